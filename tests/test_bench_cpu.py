"""Host-side pieces of bench.py: the algorithmic work model behind the roofline
lines, the roofline arithmetic, the traffic lookup guard and the ESS estimator."""
import json
import math

import numpy as np
import pytest

import bench


W32 = {"dtype": "f32"}


@pytest.mark.parametrize("mode,kind", [
    ("per_chain", "reduce"), ("per_chain", "apply"), ("per_chain_sqrt", "reduce"), ("per_chain_sqrt", "apply"),
    ("shared", "cov_reduce"), ("shared", "cov_scan"), ("shared", "cov_apply"), ("shared", "cov_products"),
    ("table_sqrt", "cov_reduce"), ("table_sqrt", "cov_scan"), ("table_sqrt", "cov_apply"),
    ("cached", "reduce"), ("cached", "apply"), ("cached", "backward"), ("cached", "bridge"),
    ("shared", "bridge_tree")])
def test_every_roofline_kind_has_positive_work(mode, kind):
    d, T, C = 30, 1024, 32
    nb, nbc = 32, 256
    flops, byt = bench.kernel_work(mode, kind, W32, d, T, C, nb, nbc, True, 4)
    assert flops is not None and flops > 0
    assert byt is None or byt > 0


def test_means_path_bytes_are_the_tables_and_vectors_once():
    d, T, C, s = 30, 1024, 32, 4
    _, byt = bench.kernel_work("cached", "apply", W32, d, T, C, 32, 256, True, s)
    tab, vec = T * d * d * s, C * T * d * s
    # forward: four tables, y~ in and U out; reverse: one table and y~*; mean of the two launches
    assert byt == (4 * tab + 2 * vec + tab + vec) / 2


def test_doubling_scan_counts_one_operator_per_prefix():
    """Doubling over the T steps: T - 1 prefix operators (C part only) plus the powers
    of all levels but the last, spread over ceil(log2 T) launches."""
    d, T = 30, 1024
    flops, _ = bench.kernel_work("shared", "cov_scan", W32, d, T, 32, 32, 256, True, 4)
    levels = math.ceil(math.log2(T))
    assert levels == 10
    assert flops == pytest.approx(((T - 1) * bench.conly_flops(d)
                                   + (levels - 1) * bench.matrix_combine_flops(d)) / levels)


def test_roofline_line_arithmetic(monkeypatch):
    # the device's SM count and maximum clock, as device_caps would read them
    monkeypatch.setattr(bench, "device_caps", lambda peaks: (152, 2000.0, "test"))
    prof = {"apply": (2.0, 4)}                       # 4 launches in 2 ms
    peaks = {"hbm_gbs": 6000.0, "sm_max_mhz": 2000.0}
    line = bench.roofline_line("cached", "apply", prof, W32, 30, 1024, 32, 32, 256, True, 4, peaks, 2, "p")
    _, byt = bench.kernel_work("cached", "apply", W32, 30, 1024, 32, 32, 256, True, 4)
    assert line["bound"] == "hbm" and line["unit"] == "GB/s"
    assert line["achieved"] == pytest.approx(byt / 0.5e-3 / 1e9)
    assert line["frac"] == pytest.approx(line["achieved"] / 6000.0)
    line = bench.roofline_line("per_chain", "apply", {"apply": (1.0, 1)}, W32, 30, 1024, 32, 32, 256, True, 4,
                               peaks, 1, "p")
    flops, _ = bench.kernel_work("per_chain", "apply", W32, 30, 1024, 32, 32, 256, True, 4)
    peak = 152 * 128 * 2 * 2000.0 * 1e6 / 1e12
    assert line["bound"] == "alu" and line["peak"] == pytest.approx(peak)
    assert line["achieved"] == pytest.approx(flops / 1e-3 / 1e12)


def test_traffic_is_used_only_for_the_captured_sources(tmp_path, monkeypatch):
    rec = {"source_sha256": "abc", "dram_bytes_per_launch": {"k_x": 123.0}}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: "abc")
    assert bench.dram_traffic("k_x") == 123.0
    assert bench.dram_traffic("k_y") is None
    monkeypatch.setattr(bench, "source_hash", lambda: "changed")
    assert bench.dram_traffic("k_x") is None


def test_source_hash_is_stable():
    assert bench.source_hash() == bench.source_hash()


def test_geyer_ess_of_white_noise_and_of_an_ar1_series():
    rng = np.random.default_rng(0)
    n = 20000
    x = rng.standard_normal(n)
    assert 0.8 * n < bench.geyer_ess(x) < 1.2 * n
    phi = 0.9
    y = np.empty(n)
    y[0] = rng.standard_normal()
    for t in range(1, n):
        y[t] = phi * y[t - 1] + rng.standard_normal()
    # integrated autocorrelation time of an AR(1): (1 + phi) / (1 - phi) = 19
    assert n / 19 * 0.7 < bench.geyer_ess(y) < n / 19 * 1.3


def test_batched_workload_and_padded_widths():
    """The batched workload: T in [128, 4096], widths cycling 8, 16, 32, 64, delta
    scaled from the calibrated d = 30, T = 1024 value; padded widths of the kernels."""
    wls = bench.batched_instances(n_inst=8)
    assert [w.d for w in wls] == [8, 16, 32, 64] * 2
    assert all(128 <= w.T <= 4096 for w in wls)
    for w in wls:
        assert abs(w.delta - 0.0183 * math.sqrt(30 * 1024 / (w.d * w.T))) < 1e-15
    assert [bench.batch_p(d) for d in (1, 4, 5, 8, 9, 30, 33, 64, 65, 128)] == [4, 4, 8, 8, 16, 32, 64, 64, 128, 128]
    with pytest.raises(ValueError):
        bench.batch_p(129)
