"""Host arithmetic of the benchmark's roofline figures (no GPU): the algorithmic work per
launch and the fractions of the peaks, checked by hand for one stencil, gather and scatter
launch in each form."""
from types import SimpleNamespace

import pytest

import bench


def _wl(Nd=1_000_000, ncol=100):
    return SimpleNamespace(Nd=Nd, ncol=ncol)


def test_fp64_stencil_roofline_counts_44_flop_per_point_orbital():
    # 10 launches of 20 ms in total: 2 ms per launch; 44 * 1e8 flop / 2e-3 s = 2.2 TFLOP/s
    r = bench.kernel_roofline("stencil", (20.0, 10), _wl(), "f64", 0)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(44 * 1e8 / 2e-3 / 1e12)
    peak = 152 * 2 * 2 * 2.07 / 1e3
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    # the count with every FMA as two flops, reported beside it
    assert r["frac_fma_as_two_flops"] == pytest.approx(59 * 1e8 / 2e-3 / 1e12 / peak)


def test_traffic_is_null_once_the_kernel_source_changed(monkeypatch):
    sha = bench._source_sha16("stencil.cu")
    monkeypatch.setitem(bench.TRAFFIC_CAPTURES, ("f32", "stencil"), (12.5, "stencil.cu", sha))
    assert bench.kernel_roofline("stencil", (6.0, 3), _wl(), "f32", 0)["traffic"] == pytest.approx(12.5 * 1e8)
    monkeypatch.setitem(bench.TRAFFIC_CAPTURES, ("f32", "stencil"), (12.5, "stencil.cu", "0" * 16))
    assert bench.kernel_roofline("stencil", (6.0, 3), _wl(), "f32", 0)["traffic"] is None


def test_fp64_gather_counts_two_flop_per_function_point_and_column():
    r = bench.kernel_roofline("gather", (4.0, 2), _wl(), "f64", 5_000_000)
    assert r["achieved"] == pytest.approx(2.0 * 5e6 * 100 / 2e-3 / 1e12)


@pytest.mark.parametrize("name,bytes_per", [("stencil", 12.0), ("gather", 4.0), ("scatter", 8.0)])
def test_float_kernels_count_their_block_bytes_against_hbm(name, bytes_per):
    r = bench.kernel_roofline(name, (6.0, 3), _wl(), "f32", 0)
    peak, _ = bench.hbm_peak()
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(bytes_per * 1e8 / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    assert r["traffic"] is None or r["traffic"] > 0


def test_whole_job_rate_counts_every_rank():
    # 4 ranks, 3 steps of 2e9 units each, 6 s on the slowest rank
    assert bench.whole_job_rate(2e9, 3, 4, 6.0) == pytest.approx(4e9)


def test_clock_sampler_reads_the_median_clock_and_the_active_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join([
        "0, 2070, 2070, 640.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 700.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]) + "\n")

    class DoneProcess:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0
    s = bench.ClockSampler(0)
    s.proc, s.path = DoneProcess(), str(path)
    out = s.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
