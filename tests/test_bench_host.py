"""Host logic of the benchmark (no GPU): the algorithmic-byte model behind the roofline
fraction, the committed ncu traffic table it reads, and the parsing of the clock samples
that decides whether a run is rejected for throttling."""
import bench


def test_algorithmic_bytes_of_the_large_workload():
    """512^3 particles on a 1024^3 mesh, 100 steps: the per-pass algorithmic bytes sum to
    about 311 GB per gradient step (one forward and one adjoint PM step), the column passes
    (the dominant category) to 90.2 GB per pair of forward and adjoint force evaluations
    (n + 1 of them per evaluation), the figure the roofline object reports."""
    n, N, M = 100, 512 ** 3, 1024 ** 3
    alg = bench.algorithmic_bytes(n, N, M)
    per_step = sum(alg.values()) / n
    assert abs(per_step / 311e9 - 1) < 0.01
    assert abs(alg["fft_cols"] / (n + 1) / 90.19e9 - 1) < 0.001
    assert bench.algorithmic_bytes(n, N, M, batch=16)["scatter"] == 16 * alg["scatter"]


def test_ncu_traffic_table_parser(tmp_path, monkeypatch):
    """The bench reads per-category DRAM bytes per PM step from the committed ncu summary's
    six-column table; the step's traffic is their sum, and a missing summary gives null."""
    f = tmp_path / "t.md"
    f.write_text("| category | a | b | c | d | bytes |\n|---|---|---|---|---|---|\n"
                 "| fft_cols | 1 | 2 | 1.0 | 3 | 8.5e10 |\n| scatter | 1 | 2 | 1.0 | 3 | 4.0e10 |\n")
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(f))
    assert bench._ncu_traffic("fft_cols") == 8.5e10
    assert bench._ncu_traffic("no_such_category") is None
    assert bench._ncu_traffic_step() == 12.5e10
    monkeypatch.setattr(bench, "TRAFFIC_SUMMARY", str(tmp_path / "absent.md"))
    assert bench._ncu_traffic_step() is None


def test_compulsory_bytes_of_the_large_workload():
    """One forward + one adjoint PM step at 512^3 particles / 1024^3 mesh moves 187.4 GB of
    compulsory traffic: the denominator of the headline roofline fraction."""
    assert abs(bench.compulsory_bytes_per_pm_step(512 ** 3, 1024 ** 3) / 187.37e9 - 1) < 1e-3


def test_clock_samples_median_and_throttle_reasons():
    cs = bench.ClockSampler(0)
    cs.proc = None
    assert cs.stop()["reasons"] == ["nvidia-smi unavailable"]

    class _Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs.proc = _Done()
    cs.lines = [
        "0, 2070, 2070, 910.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2040, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 905.3, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    out = cs.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    cs.lines = ["0, 1500, 2070, 800, 0x8, Not Active, Active, Not Active, Not Active"]
    assert cs.stop()["reasons"] == ["hw_thermal_slowdown"]
