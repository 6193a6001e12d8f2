"""CPU tests of the telemetry sampler (the paper's start / timestamp / stop /
parse monitor, Sec. 2) against a fake NVML library built here from
tests/fake_nvml/fake_nvml.c: sampled values, period, events, CSV round trip,
phase summary, error paths, and that no NVML setter is ever called."""
import ctypes
import os
import subprocess
import time

import numpy as np
import pytest

from paper_2605_13928_b300 import _lib as L
from paper_2605_13928_b300 import build as B
from paper_2605_13928_b300 import monitor

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def fake(tmp_path_factory):
    B.build()
    so = str(tmp_path_factory.mktemp("nvml") / "libfake_nvml.so")
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so,
                           os.path.join(HERE, "fake_nvml", "fake_nvml.c")])
    lib = ctypes.CDLL(so)
    lib.fake_nvml_calls.restype = ctypes.c_int
    lib.fake_nvml_calls.argtypes = [ctypes.c_char_p]
    old = os.environ.get("TSNE_NVML_LIB")
    os.environ["TSNE_NVML_LIB"] = so
    yield lib
    if old is None:
        os.environ.pop("TSNE_NVML_LIB", None)
    else:
        os.environ["TSNE_NVML_LIB"] = old


def test_sampling_events_csv_and_summary(fake, tmp_path):
    path = str(tmp_path / "trace.csv")
    u0 = fake.fake_nvml_calls(b"util")
    mon = monitor.Monitor.start(period=0.01, device=0, csv=path)
    mon.timestamp("phase_a")
    time.sleep(0.15)
    mon.timestamp("phase_b")
    time.sleep(0.15)
    mon.stop()
    mon.stop()  # idempotent
    with pytest.raises(L.TsneError):
        mon.timestamp("after_stop")
    tr = mon.parse()
    n = len(tr.samples["t"])
    assert 10 <= n <= 60, n  # 0.3 s at a 10 ms period
    assert fake.fake_nvml_calls(b"util") - u0 == n
    s = tr.samples
    assert np.all(np.diff(s["t"]) > 0)
    assert np.all(s["gpu_util"] == (np.arange(u0, u0 + n) % 101))
    assert np.all(s["mem_util"] == 37) and np.all(s["mem_used_mb"] == 3 * 1024)
    assert np.all(s["temp_c"] == 41) and np.all(s["sm_mhz"] == 2032)
    assert np.all(s["power_w"] == -1)  # the fake's power query fails
    assert [e[1] for e in tr.events] == ["phase_a", "phase_b"]
    assert 0.12 < tr.events[1][0] - tr.events[0][0] < 1.0
    assert fake.fake_nvml_calls(b"set") == 0
    # the CSV holds the same trace (6 decimals of time)
    tc = monitor.parse_csv(path)
    assert [e[1] for e in tc.events] == ["phase_a", "phase_b"]
    for c in monitor.COLUMNS[1:]:
        assert np.array_equal(tc.samples[c], s[c]), c
    assert np.allclose(tc.samples["t"], s["t"], atol=1e-6)
    summ = tr.summary()
    assert [p["phase"] for p in summ] == ["phase_a", "phase_b"]
    assert all(p["samples"] >= 5 for p in summ)
    assert summ[0]["temp_c"] == 41 and summ[0]["power_w"] is None
    mon.close()
    assert fake.fake_nvml_calls(b"shutdown") >= 1


def test_context_manager_and_counts(fake):
    with monitor.Monitor.start(period=0.005) as mon:
        time.sleep(0.05)
        mon.timestamp("x")
    lib = L.lib()
    assert lib.tsne_mon_count(mon._h, 0) >= 3
    assert lib.tsne_mon_count(mon._h, 1) == 1
    mon.close()


def test_error_paths(fake, monkeypatch):
    lib = L.lib()
    err = ctypes.c_int(0)
    assert not lib.tsne_mon_start(1, 0.1, None, ctypes.byref(err)) and err.value == -1  # no device 1
    assert not lib.tsne_mon_start(0, 0.0, None, ctypes.byref(err)) and err.value == -1  # period
    assert not lib.tsne_mon_start(-1, 0.1, None, ctypes.byref(err)) and err.value == -1
    assert not lib.tsne_mon_start(0, 0.1, b"/nonexistent_dir/x.csv", ctypes.byref(err))
    assert err.value == -1
    monkeypatch.setenv("FAKE_NVML_FAIL_INIT", "1")
    assert not lib.tsne_mon_start(0, 0.1, None, ctypes.byref(err)) and err.value == -7
    monkeypatch.delenv("FAKE_NVML_FAIL_INIT")
    monkeypatch.setenv("TSNE_NVML_LIB", "/nonexistent/libnvidia-ml.so.1")
    with pytest.raises(L.TsneError) as e:
        monitor.Monitor.start(period=0.1)
    assert e.value.code == -7
    assert lib.tsne_mon_mark(None, b"x") == -1 and lib.tsne_mon_stop(None) == -1
    lib.tsne_mon_free(None)
    assert fake.fake_nvml_calls(b"set") == 0
