"""Host-side logic of bench.py: the per-kernel table and the roofline object (no GPU)."""
import pytest

import bench

PEAKS = {"hbm_gbs": 6686.1, "bf16_tflops": 1925.2}
ALU = {"fp64": 1.06, "fp32": 78.4}


def _kern():
    # per step: launches, summed milliseconds, algorithmic bytes and flops
    return {
        "coarse_gmres": {"launches": 30, "ms": 20.0, "bytes": 1.0e8, "flops": 0.0},
        "dslash_proj": {"launches": 260, "ms": 13.0, "bytes": 260 * 172e6, "flops": 260 * 8e8},
        "galerkin_tc": {"launches": 1, "ms": 4.4, "bytes": 1.6e9, "flops": 1.45e10,
                        "issued_flops": 4.2e14 * 4.4e-3},
        "svd_gram_df64": {"launches": 5, "ms": 2.8, "bytes": 1.9e9, "flops": 3.0e12 * 2.8e-3},
        "svd_jacobi_df64": {"launches": 4, "ms": 2.2, "bytes": 3.5e7, "flops": 0.0},
        "dslash_c128": {"launches": 3, "ms": 0.7, "bytes": 3 * 126e6, "flops": 3 * 1.73e8},
        "idle": {"launches": 1, "ms": 0.0, "bytes": 0.0, "flops": 0.0},
    }


def test_dominant_kernel_roofline():
    kernels, roof = bench.kernel_table(_kern(), ALU, PEAKS, "measured")
    # coarse_gmres takes longer but is latency-bound (no peak): the roofline is dslash_proj's
    assert roof["kernel"] == "dslash_proj"
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and roof["peak"] == PEAKS["hbm_gbs"]
    per_launch_s = 13.0e-3 / 260
    assert roof["achieved"] == pytest.approx(172e6 / per_launch_s / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(172e6)
    # the ncu traffic recorded for this kernel on the bench workload, or None if none is
    assert roof["traffic"] == bench.NCU_TRAFFIC.get(("dslash_proj", bench.WORKLOAD))
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof


def test_each_kernel_against_its_own_unit():
    kernels, _ = bench.kernel_table(_kern(), ALU, PEAKS, "measured")
    assert abs(sum(k["share"] for k in kernels.values()) - 1) < 1e-12
    assert list(kernels)[0] == "coarse_gmres"                    # sorted by time
    assert kernels["coarse_gmres"]["bound"] == "latency" and kernels["coarse_gmres"]["frac"] is None
    assert kernels["svd_jacobi_df64"]["frac"] is None
    # the method's FP64-equivalent flops against the double-float (FP32 / 12) staging peak;
    # the bf16 digit-plane products it issues against the bf16 tensor peak, as extra fields
    assert kernels["galerkin_tc"]["bound"] == "alu"
    assert kernels["galerkin_tc"]["frac"] == pytest.approx(1.45e10 / 4.4e-3 / 1e12 / (ALU["fp32"] / 12))
    assert kernels["galerkin_tc"]["tensor_issued_TFLOPs"] == pytest.approx(420.0)
    assert kernels["galerkin_tc"]["tensor_issued_frac_of_bf16"] == pytest.approx(420.0 / PEAKS["bf16_tflops"])
    assert kernels["svd_gram_df64"]["bound"] == "alu"
    assert kernels["svd_gram_df64"]["frac"] == pytest.approx(3.0 / (ALU["fp32"] / 12))
    assert kernels["dslash_c128"]["bound"] == "alu"
    assert kernels["dslash_c128"]["frac"] == pytest.approx(1.73e8 / (0.7e-3 / 3) / 1e12 / ALU["fp64"])
    assert "frac" not in kernels["idle"]


def test_tensor_kernel_dominant_and_empty_table():
    k = {"galerkin_tc": {"launches": 1, "ms": 5.0, "bytes": 1e9, "flops": 1e12}}
    _, roof = bench.kernel_table(k, ALU, PEAKS, "measured")
    assert roof["unit"] == "TFLOP/s"
    assert roof["traffic"] == bench.NCU_TRAFFIC.get(("galerkin_tc", bench.WORKLOAD))
    assert roof["achieved"] == pytest.approx(1e12 / 5e-3 / 1e12)
    assert bench.kernel_table({}, ALU, PEAKS, "measured") == ({}, None)
    only_latency = {"coarse_gmres": {"launches": 1, "ms": 1.0, "bytes": 1.0, "flops": 0.0}}
    kernels, roof = bench.kernel_table(only_latency, ALU, PEAKS, "measured")
    assert roof is None and kernels["coarse_gmres"]["frac"] is None


def test_config_object_is_shared_by_both_arms():
    cfg = bench.workload()
    c = bench.bench_config(cfg, 1)
    assert c["workload"] == bench.WORKLOAD and c["dims"] == [16, 16, 16, 32]
    assert c["parallelism"] == "single" and bench.bench_config(cfg, 4)["parallelism"] == "replicas"
