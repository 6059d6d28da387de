"""Host logic of bench.py on CPU: the clock-record parser, the algorithmic work counted per
kernel launch (checked against closed forms of the same sums), the DRAM-traffic scaling, the
single-rank throughput and the reference arm's JSON line.  No GPU."""
import math

import pytest

import bench


class _FakeSmi:
    """Stands in for the nvidia-smi sampler process: returns a fixed CSV record."""

    def __init__(self, text):
        self.text = text
        self.terminated = False

    def terminate(self):
        self.terminated = True

    def communicate(self, timeout=None):
        return self.text, ""

    def kill(self):
        pass


def test_clock_summary_parses_samples_of_one_gpu():
    rec = "\n".join([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1950, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "1, 300, 2070, 100.0, 0x0, Active, Not Active, Not Active, Not Active",  # other GPU
        "0, 2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    p = _FakeSmi(rec)
    s = bench._clock_summary(p, 0)
    assert p.terminated
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2010.0
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # GPU 1's hw_slowdown is not this run's
    assert bench._clock_summary(None, 0) is None
    assert bench._clock_summary(_FakeSmi(""), 0) is None


PEAKS = {"hbm_gbs": 6756.2, "bf16_tflops": 1914.9, "bf16_tflops_sustained": 1713.5,
         "sm_max_mhz": 2070.0}


@pytest.mark.parametrize("n", [1024, 16384])
def test_update_work_is_the_left_looking_sum(n):
    """k_oz_update: the method's work is the left-looking update, sum over block columns j of
    (n - 64 j) x 64 x (64 j) multiply-adds, which for n a multiple of 64 is (n^3 - 64^2 n) / 6
    (2 flops each, ~n^3/3); the tensor pipe runs 21 BF16 digit products per multiply-add, which
    the separate issue fraction counts."""
    ms = 10.0
    r = bench.kernel_rooflines({"k_oz_update": (ms, 100)}, "mixed", n, 20000, PEAKS,
                               "measured", steps=1)
    (u,) = r
    mac = (n ** 3 - 64 ** 2 * n) // 6
    assert bench.chol_update_macs(n) == mac
    assert u["achieved"] == pytest.approx(2 * mac / (ms * 1e-3) / 1e12, rel=1e-12)
    assert u["peak"] == PEAKS["bf16_tflops_sustained"]
    assert u["frac"] == pytest.approx(u["achieved"] / u["peak"], rel=1e-12)
    assert u["mma_issue_frac"] == pytest.approx(21 * u["frac"], rel=1e-12)
    assert u["work_flops_per_step"] == 2 * mac
    assert u["launch_ms"] == pytest.approx(ms / 100)
    assert u["bound"] == "tensor" and u["unit"] == "TFLOP/s"


@pytest.mark.parametrize("n,paths", [(9216, 20096), (16384, 20000)])
def test_sweep_work_is_the_limit_gemm(n, paths):
    """k_sov_tc: the method's work is the limit GEMM, n (n - 1) flops per path; the far part on
    the tensor cores covers every entry of L left of the 128 x 128 diagonal blocks,
    n (n - 128) / 2 multiply-adds per path for 128-path tiles, 3 FP16 MMAs each (issue
    fraction)."""
    ms, launches = 40.0, 2
    r = bench.kernel_rooflines({"k_sov_tc": (ms, launches)}, "mixed", n, paths, PEAKS,
                               "measured", steps=launches)
    (s,) = r
    assert s["achieved"] == pytest.approx(n * (n - 1) * paths * launches / (ms * 1e-3) / 1e12,
                                          rel=1e-12)
    tiles = math.ceil(paths / 128)
    mac = tiles * 128 * n * (n - 128) // 2
    assert bench.sweep_far_macs(n, tiles) == mac
    issue = 2 * 3 * mac * launches / (ms * 1e-3) / 1e12
    assert s["mma_issue_frac"] == pytest.approx(issue / PEAKS["bf16_tflops_sustained"], rel=1e-12)
    assert s["work_flops_per_launch"] == n * (n - 1) * paths
    hv = s["hbm_view"]
    per_launch_s = ms * 1e-3 / launches
    assert hv["achieved"] == pytest.approx(s["traffic"] / per_launch_s / 1e9, rel=1e-12)
    assert hv["frac"] == pytest.approx(hv["achieved"] / PEAKS["hbm_gbs"], rel=1e-12)


def test_simt_and_fp64_work():
    n, paths = 256, 200000
    r = bench.kernel_rooflines({"k_sov_simt_f64": (30.0, 1), "k_syrk": (5.0, 3)}, "fp64", n,
                               paths, PEAKS, "measured", steps=1)
    by = {x["kernel"]: x for x in r}
    assert by["k_sov_simt_f64"]["achieved"] == pytest.approx(
        n * (n - 1) * paths / 30e-3 / 1e12, rel=1e-12)
    # three of the (n/64 - 1) = 3 trailing updates of one factorisation: n^3/3 flops
    assert by["k_syrk"]["achieved"] == pytest.approx(n ** 3 / 3 / 5e-3 / 1e12, rel=1e-12)
    assert all(x["bound"] == "alu" and x["traffic"] is None for x in r)


def test_traffic_scaling_reproduces_the_measured_case():
    for k, v in bench.TRAFFIC_BYTES0.items():
        assert bench._traffic(k, bench.TRAFFIC_N0, bench.TRAFFIC_TILES0) == pytest.approx(v)
    # the sweep's Y re-reads grow as n^2 x path tiles, the update's reads as n^2
    assert bench._traffic("k_sov_tc", 2 * bench.TRAFFIC_N0, 2 * bench.TRAFFIC_TILES0) == \
        pytest.approx(8 * bench.TRAFFIC_BYTES0["k_sov_tc"])
    assert bench._traffic("k_oz_update", 2 * bench.TRAFFIC_N0, 1) == \
        pytest.approx(4 * bench.TRAFFIC_BYTES0["k_oz_update"])
    assert bench._traffic("k_matern", 100, 1) is None


def test_single_rank_throughput():
    ms, v = bench.job_time_and_value(109.1, 16384 * 20000, 1)
    assert ms == 109.1
    assert v == pytest.approx(16384 * 20000 / 0.1091)


def test_reference_arm_line(monkeypatch, capsys):
    """`bench.py --impl reference` prints one JSON line with the keys the bench contract asks
    of the reference arm (here on a 16 x 16 grid instead of the 128 x 128 one, to stay fast)."""
    import json
    import types

    from paper_2405_14892_gb300 import inputs

    def small_workload(grid=0):
        w = dict(inputs.WORKLOADS["W2"], g=16, name="sov-n256-matern32-test")
        c = inputs.grid_coords(16)
        a, b = inputs.limits_for(w, c.shape[0])
        return w, c, a, b

    monkeypatch.setattr(bench, "workload", small_workload)
    monkeypatch.delenv("RANK", raising=False)
    bench.run_reference(types.SimpleNamespace(steps=2, warmup=1, gpus=1))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == bench.UNIT and d["metric"] == bench.METRIC
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 2
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert "16 of 20000 paths at n=256" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == "sov-n256-matern32-test"
