"""Host logic of the measurement (bench.py): the launch filter behind the matvec roofline, the
roofline arithmetic and the choice of the dominant kernel, and the JSON line's defaults. CPU
only: no kernels run."""
import importlib.util
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_working_launches_sets_aside_early_exits(bench):
    # 40 launches that streamed the operator (70-80 us) and 6 that exited at once (3 us)
    rng = np.random.default_rng(0)
    streamed = list(0.070 + 0.010 * rng.random(40))
    d = streamed[:20] + [0.003] * 6 + streamed[20:]
    ms, working, skipped = bench._working_launches(d)
    assert (working, skipped) == (40, 6)
    assert ms == pytest.approx(sum(streamed))
    assert bench._working_launches([]) == (0.0, 0, 0)
    # all launches alike: none set aside
    assert bench._working_launches([0.05] * 7)[1:] == (7, 0)


def test_roofline_arithmetic_and_dominant_kernel(bench):
    n = 10240
    ld = (n + 31) // 32 * 32
    kern = {"gemv": (40.0, 500), "gemv_bf16": (120.0, 1600), "assemble_regular": (76.8, 64)}
    working = {"gemv": (40.0, 500, 0), "gemv_bf16": (118.0, 1500, 100)}
    peaks = {"hbm_gbs": 6672.5, "sm_max_mhz": 2070.0}
    dom, table = bench.roofline({"n": n, "measured": kern, "working": working}, peaks, "measured")
    assert dom == "gemv_bf16"  # the most device time
    b = table["gemv_bf16"]
    bytes_per = 4.0 * n * ld + 8.0 * ld + 16.0 * n
    assert b["algorithmic_bytes_per_launch"] == bytes_per
    assert b["achieved"] == pytest.approx(bytes_per / (118.0 / 1500 * 1e-3) / 1e9)
    assert b["frac"] == pytest.approx(b["achieved"] / 6672.5)
    assert (b["launches"], b["launches_exited_early"]) == (1500, 100)
    a = table["assemble_regular"]
    fp32_peak = 128 * 152 * 2 * 2070.0e6 / 1e12
    assert a["peak"] == pytest.approx(fp32_peak)
    assert a["achieved"] == pytest.approx(float(n) * n * bench.FLOPS_PER_PAIR / (76.8 / 64 * 1e-3) / 1e12)
    assert a["bound"] == "alu" and b["bound"] == "hbm"


def test_peaks_fall_back_when_unmeasured(bench, tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, kind = bench._peaks()
    assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0 and peaks["bf16_tflops"] == 1900.0


def test_sustained_rate_uses_the_streams_own_rate(bench):
    """A seeded Poisson stream's mean rate differs from the nominal one: the server is judged
    against the rate the stream actually offered, and a growing queue fails it."""
    # 300 requests whose last arrival is at 6.92 s offer 43.4 req/s; 42.7 served/s keeps up
    offered, served, ok = bench._sustained(300, 6.915, 300 / 42.7, 339.0, 283.0)
    assert abs(offered - 300 / 6.915) < 1e-12 and abs(served - 42.7) < 1e-9 and ok
    # the same completions against a stream that really offered 50 req/s do not
    assert not bench._sustained(300, 6.0, 300 / 42.7, 339.0, 283.0)[2]
    # keeping up on average while the last third waits twice as long as the first: a growing queue
    assert not bench._sustained(300, 6.915, 300 / 43.0, 300.0, 600.0)[2]
