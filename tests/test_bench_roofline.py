"""The benchmark's roofline bookkeeping on CPU: per-operation timings are
grouped by the CUDA kernel that runs them, the dominant kernel is reported
against its own bound, the tensor-core kernel beside it, and the measured
DRAM traffic is attached only for the configuration it was captured on."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PEAKS = {"hbm_gbs": 6762.3, "bf16_tflops": 1906.8, "bf16_tflops_sustained": 1713.1,
         "sm_max_mhz": 2070.0}


def _st(launches, ms, flops, nbytes):
    return {"launches": launches, "ms": ms, "flops": flops, "bytes": nbytes}


def test_every_operation_label_belongs_to_one_kernel_family():
    seen = {}
    for fam, (names, bound) in bench.KERNEL_FAMILIES.items():
        assert bound in ("hbm", "tensor", "alu")
        for nm in names:
            assert nm not in seen, (nm, fam, seen.get(nm))
            seen[nm] = fam
    # the labels the engine emits for the tensor-core routes
    assert seen["contract_tc_tf32"] == "k_tc_gemm"
    assert seen["contract_tc_direct_tf32"] == "k_tc_gemm_direct"
    assert seen["contract_outer_c64"] == "k_outer"


def test_dominant_hbm_kernel_reported_against_measured_bandwidth():
    stats = {
        # 10 launches moving 500 MB each in 0.2 ms: 2.5 TB/s
        "contract_tc_direct_tf32": _st(10, 2.0, 1e12, 10 * 500e6),
        "contract_tc_tf32": _st(4, 1.0, 4 * 2e11, 4 * 400e6),
        "combine": _st(20, 1.5, 0.0, 20 * 100e6),
    }
    rl, dom = bench.roofline_of(stats, PEAKS, "measured", "tf32", 2)
    assert dom == "k_tc_gemm_direct"
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert abs(rl["achieved"] - 2500.0) < 1.0
    assert abs(rl["frac"] - 2500.0 / 6762.3) < 1e-3
    assert rl["launches"] == 10 and abs(rl["avg_launch_us"] - 200.0) < 1e-6
    assert abs(rl["share_of_step"] - 2.0 / 4.5) < 1e-4
    # the traffic of a kernel is reported only while its counters are current
    assert rl["traffic"] == bench.MEASURED_TRAFFIC.get(("k_tc_gemm_direct", "tf32", 2))
    # the tcgen05 short-sum kernel rides along against the TF32 tensor peak
    tk = rl["tensor_kernel"]
    assert tk["kernel"] == "k_tc_gemm" and tk["bound"] == "tensor"
    assert abs(tk["peak"] - 1713.1 * 1.1 / 2.25) < 0.1
    assert abs(tk["achieved"] - 800.0) < 0.01  # 8e11 flop in 1 ms


def test_traffic_only_for_the_captured_configuration():
    stats = {"contract_tc_direct_tf32": _st(10, 2.0, 1e12, 5e9)}
    rl, _ = bench.roofline_of(stats, PEAKS, "measured", "bf16", 2)
    assert rl["traffic"] is None
    rl, _ = bench.roofline_of(stats, PEAKS, "measured", "tf32", 3)
    assert rl["traffic"] is None


def test_alu_kernel_peak_from_unit_counts_and_clock():
    stats = {"contract_simt_c64": _st(100, 4.0, 40e12 * 4e-3, 1e9)}
    rl, dom = bench.roofline_of(stats, PEAKS, "measured", "fp32", 2)
    assert dom == "k_contract" and rl["bound"] == "alu"
    assert abs(rl["peak"] - 152 * 128 * 2 * 2070e6 / 1e12) < 0.01
    assert abs(rl["achieved"] - 40.0) < 1e-6
