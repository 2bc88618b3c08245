"""Host logic of bench.py's roofline accounting (no GPU): the per-class
algorithmic work of the scope table, the dominant class, the contract's
bound vocabulary, and the DRAM-traffic guard on the kernels' sources."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

DIMS = {"nao": 512, "nocc": 71, "nvir": 441, "nJ": 102, "nK": 42}


def _stats(**kw):
    st = {"tc_gemm_ms": 5.7, "tc_gemm_flops": 2.3e11, "gemm_ms": 3.0, "gemm_flops": 1.0e9,
          "emu_gemm_ms": 2.2, "emu_gemm_flops": 8.6e9, "ff_gemm_ms": 1.2, "ff_gemm_flops": 1.3e9,
          "contract_ms": 1.9, "contract_bytes": 3.5e9, "eig_ms": 2.5, "int3c_ms": 0.9,
          "int3c_deriv_ms": 7.8}
    st.update(kw)
    return st


def test_mixed_work_split_and_dominant_class():
    nov = DIMS["nocc"] * DIMS["nvir"]
    alg = bench.algorithmic_work("mixed", DIMS, 75, 19)
    # the Coulomb part of A.X is the double-FP32 class's work, not the FP64 class's
    assert alg["ff_gemm_f64x"] == 4.0 * nov * DIMS["nJ"] * 75
    assert alg["dgemm_fp64"] == 2.0 * DIMS["nocc"] ** 2 * DIMS["nao"] * DIMS["nK"]
    roof, table = bench.classify(_stats(), 1, 23.7, "mixed", DIMS, 75, 19)
    assert roof["kernel"] == "tc_gemm_3xtf32"  # largest time, side-stream integrals excluded
    assert roof["bound"] == "tensor" and roof["pipe"] == "tensor (tf32)"
    assert 0 < roof["frac"] < 1 and roof["unit"] == "TFLOP/s"
    assert table["contract"]["unit"] == "GB/s" and table["contract"]["bound"] == "hbm"
    assert table["ff_gemm_f64x"]["bound"] == "fp32 fma (double-FP32)"


def test_fp64_form_is_alu_bound_on_its_gemms():
    st = _stats(tc_gemm_ms=0.0, emu_gemm_ms=0.0, ff_gemm_ms=0.0, gemm_ms=284.0, gemm_flops=2.9e11)
    roof, _ = bench.classify(st, 1, 302.0, "fp64", DIMS, 118, 19)
    assert roof["kernel"] == "dgemm_fp64" and roof["bound"] == "alu"
    assert roof["traffic"] is None  # the traffic table is for the mixed form


def test_traffic_guard_follows_the_source():
    t = bench.TRAFFIC["tc_gemm_3xtf32"]
    assert bench.traffic_for("tc_gemm_3xtf32") in (None, t["bytes_per_eval"])
    saved = t["sha"]
    try:
        t["sha"] = "0" * 16  # a changed kernel source invalidates the counters
        assert bench.traffic_for("tc_gemm_3xtf32") is None
    finally:
        t["sha"] = saved
