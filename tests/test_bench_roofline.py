"""Host logic of bench.py's roofline entry (CPU only).

The entry names the roof that binds a kernel family: for the tensor-core
families the lower of the TF32 roof (a third of the peak, three MMA passes
per product) and arithmetic intensity x HBM; the double-single families of
the FP32 mode are held to the FP32-pipe rate of a double-single multiply-add.
"""
import math

import bench

HBM = 6678.5  # GB/s


def test_streaming_block_solve_is_held_to_hbm():
    # 4.6 flop per byte: 4.6 * 6.68 TB/s = 31 TFLOP/s, far below the TF32 roof
    rec = {"ms": 100.0, "flops": 4.6e11, "bytes": 1.0e11, "launches": 10}
    r = bench.family_roofline("eig_solve", rec, "mixed", HBM, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert math.isclose(r["achieved"], 1.0e11 / 0.1 / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / HBM)
    assert math.isclose(r["flop_per_byte"], 4.6)


def test_dense_factorisation_is_held_to_the_tensor_roof():
    # 1000 flop per byte: intensity x HBM is above a third of the TF32 peak
    rec = {"ms": 10.0, "flops": 1.0e12, "bytes": 1.0e9, "launches": 1}
    r = bench.family_roofline("factor", rec, "mixed", HBM, "measured")
    assert r["bound"] == "tensor" and r["unit"] == "TFLOP/s"
    peak, _ = bench.tf32_peak()
    assert math.isclose(r["frac"], (1.0e12 / 0.01) / peak)


def test_fp64_mode_factorisation_is_fp64_alu():
    rec = {"ms": 10.0, "flops": 1.0e10, "bytes": 1.0e9, "launches": 1}
    r = bench.family_roofline("factor", rec, "fp64", HBM, "measured")
    assert r["bound"] == "alu"
    assert math.isclose(r["peak"], bench.fp64_peak() / 1e12)


def test_double_single_families_use_their_derived_peak():
    assert math.isclose(bench.ds_peak(), 152 * 128 / 12 * 2 * 2070e6)
    rec = {"ms": 50.0, "flops": 1.0e11, "bytes": 1.0e10, "launches": 5}
    for fam in ("spmm", "gram", "gemm"):
        r = bench.family_roofline(fam, rec, "mixed", HBM, "measured")
        assert r["bound"] == "alu"
        assert math.isclose(r["peak"], bench.ds_peak() / 1e12)
        assert math.isclose(r["frac"], (1.0e11 / 0.05) / bench.ds_peak())
        # FP64 mode: the same families are FP64-pipe bound
        r64 = bench.family_roofline(fam, rec, "fp64", HBM, "measured")
        assert math.isclose(r64["peak"], bench.fp64_peak() / 1e12)


def test_hbm_families_report_bandwidth():
    rec = {"ms": 2.0, "flops": 0.0, "bytes": 9.23e9, "launches": 1}
    r = bench.family_roofline("local_solve", rec, "mixed", HBM, "measured")
    assert r["bound"] == "hbm"
    assert math.isclose(r["achieved"], 9.23e9 / 0.002 / 1e9)


def test_local_solve_traffic_scaled_from_the_capture():
    # the mixed local solve carries the DRAM bytes of its ncu capture, scaled
    # by the launch's algorithmic bytes; other families report none
    rec = {"ms": 100.0, "flops": 1.0e11, "bytes": 60 * 9.23e9, "launches": 60}
    r = bench.family_roofline("local_solve", rec, "mixed", HBM, "measured")
    m = bench.MEASURED_TRAFFIC[("local_solve", "mixed")]
    ratio = m["dram_bytes_per_launch"] / m["algorithmic_bytes_per_launch"]
    assert math.isclose(r["traffic"], ratio * 9.23e9)
    assert 0.9 < ratio < 1.2
    assert bench.family_roofline("spmv", rec, "mixed", HBM, "measured")["traffic"] is None
    assert bench.family_roofline("local_solve", rec, "fp64", HBM, "measured")["traffic"] is None
