"""bench.py's roofline arithmetic against the per-site figures it reports
(algorithmic bytes and flops per site), and the kernel names it reports
against the CUDA sources."""

import glob
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_per_site_figures():
    # Dirac: spinor in + out (12 complex each) + 4 links (9 complex) + clover (36 complex slots)
    assert bench.bytes_dirac_site("fp32") == 2 * 96 + 576 == 768
    assert bench.bytes_dirac_site("bf16") == 2 * 96 + 288 == 480
    assert bench.bytes_dirac_site("fp64") == 2 * 192 + 1152
    # Schwarz colour pass per site of the colour: b, z, halo z read and z written, + fields
    assert bench.bytes_sap_site("bf16") == 4 * 96 + 288 == 672
    assert bench.bytes_sap_site("fp32") == 4 * 96 + 576 == 960
    # flops: residual + n_MR block MR steps
    assert bench.flops_sap_site(4) == 9312.0
    assert abs(bench.FP32_PEAK_TFLOPS - 80.54784) < 1e-9
    assert abs(bench.SAP_DRAM_BYTES_PER_UNIT[0] - 422.9) < 0.1 and abs(bench.SAP_DRAM_BYTES_PER_UNIT[3] - 400.7) < 0.1


def test_reported_kernel_names_exist():
    src = "".join(open(f).read() for f in glob.glob(os.path.join(ROOT, "paper_1202_2462_gb300", "csrc", "*.cu")))
    for family, names in bench.FAMILY_KERNELS.items():
        found = re.findall(r"[a-z0-9_]+_kernel|[a-z0-9_]+_partial", names)
        assert found, family
        for name in found:
            # a __global__ function of that name (launch bounds and line breaks in between)
            assert re.search(r"__global__[^;{]*?\b" + name + r"\s*\(", src, re.S), (family, name)


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_summary():
    """The clocks summary of the bench line from nvidia-smi's CSV rows (index,
    SM MHz, max SM MHz, power, active mask, then the four reasons): median SM
    clock under load, the maximum, and every throttle reason seen active."""
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.proc = _DoneProcess()
    cs.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1100.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = cs.stop()
    assert out["sm_mhz"] == 2070 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    cs.lines = ["0, 1500, 2070, 800, 0x8, Active, Not Active, Active, Not Active"]
    out = cs.stop()
    assert out["sm_mhz"] == 1500 and out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
