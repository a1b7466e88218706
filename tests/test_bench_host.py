"""Host-side logic of bench.py, on the CPU: the roofline object of a kernel
(achieved = declared algorithmic work / event time, peak by the bound,
DRAM traffic scaled from the ncu capture) and the parsing of the clock
samples taken during the timed region."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

PK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2000.0}


def test_tensor_roofline_and_scaled_traffic():
    ks = {"ms": 100.0, "launches": 10, "flops": 20e12, "bytes": 0.0}
    r = bench.roofline_of("gemm_tc3xtf32@fillin", ks, PK, 400.0)
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    assert r["achieved"] == pytest.approx(200.0)                       # 20e12 flops in 0.1 s
    assert r["peak"] == pytest.approx(1700.0 * 1.1 / 2.25 / 3.0)        # split 3xTF32 of sustained bf16
    assert r["frac"] == pytest.approx(200.0 / r["peak"])
    assert r["share"] == pytest.approx(0.25)
    assert r["algorithmic_per_launch"] == pytest.approx(2e12)
    per = bench.NCU_TRAFFIC["gemm_tc3xtf32@fillin"]["per_unit"]
    assert r["traffic"] == pytest.approx(per * 2e12)


def test_hbm_alu_and_fp64_rooflines():
    hbm = bench.roofline_of("symv_pairs_df@mv_near", {"ms": 10.0, "launches": 1, "flops": 0.0, "bytes": 50e9},
                            PK, 10.0)
    assert hbm["bound"] == "hbm" and hbm["achieved"] == pytest.approx(5000.0) and hbm["peak"] == 6800.0
    assert hbm["traffic"] == pytest.approx(bench.NCU_TRAFFIC["symv_pairs_df@mv_near"]["per_unit"] * 50e9)
    alu = bench.roofline_of("getrf_f32@fillin", {"ms": 1000.0, "launches": 2, "flops": 4e12, "bytes": 0.0}, PK, 1.0)
    assert alu["bound"] == "alu" and alu["achieved"] == pytest.approx(4.0)
    assert alu["peak"] == pytest.approx(152 * 128 * 2 * 2000e6 / 1e12)
    assert alu["traffic"] is None
    f64 = bench.roofline_of("trsm_f64@basis", {"ms": 1000.0, "launches": 1, "flops": 0.5e12, "bytes": 0.0}, PK, 1.0)
    assert f64["bound"] == "alu" and f64["peak"] == pytest.approx(1.25 * 2000.0 / 2070.0)


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_median_and_throttle_reasons():
    c = bench.ClockSampler(0)
    c.proc = _Proc()
    c.rows = [["2070", "2070", "900", "Not Active", "Not Active", "Not Active", "Not Active"],
              ["2055", "2070", "1300", "Not Active", "Not Active", "Not Active", "Active"],
              ["2070", "2070", "1350", "Not Active", "Not Active", "Not Active", "Active"],
              ["[N/A]", "2070", "0", "", "", "", ""]]
    out = c.stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_sampler_without_nvidia_smi():
    c = bench.ClockSampler(0)
    out = c.stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]
