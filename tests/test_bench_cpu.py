"""Host logic of bench.py without a GPU: workload selection (including the
@rule override), the roofline arithmetic of the reported line, and the
descriptive config fields."""
import pytest

import bench


def test_workloads_and_rule_override():
    w = bench.workload("heis2d_10x10")
    assert (w["N"], w["M"], w["chains"], w["per_chain"], w["rule"]) == (100, 200, 1024, 8, "exchange")
    h = bench.workload("heis2d_10x10@hamiltonian")
    assert h["rule"] == "hamiltonian" and h["name"] == "heis2d_10x10@hamiltonian" and h["M"] == 200
    j = bench.workload("j1j2_10x10")
    assert j["ham"]["n_edges2"] == 200 and j["ham"]["edges"].shape == (400, 2)
    assert "J1-J2" in bench.ham_text(j["ham"]) and bench.ham_text(w["ham"]) == "heis"
    with pytest.raises(AssertionError):
        bench.workload("heis2d_10x10@metropolis")


def test_roofline_of_an_alu_class():
    """Ratio terms count one FMA and one multiply: 2 flops each, against the
    FP32 lanes for the mixed path and the FP64 pipe for the FP64 path."""
    prof = {"sweep": (20.0, 4, 5e11, 5e11), "eloc": (5.0, 4, 1e11, 1e11)}
    rf, cls = bench.roofline(prof, 2, "mixed")
    assert cls == "sweep" and rf["bound"] == "alu"
    assert rf["achieved"] == pytest.approx(2 * 5e11 / 0.020 / 1e12)
    assert rf["frac"] == pytest.approx(rf["achieved"] / bench.FP32_PEAK_TFLOPS)
    assert rf["avg_launch_ms"] == pytest.approx(5.0)
    rf64, _ = bench.roofline(prof, 2, "f64")
    assert rf64["peak"] == bench.FP64_PEAK_TFLOPS


def test_roofline_of_the_tensor_class_with_traffic():
    """The tensor-core classes are rated by the method's algorithmic flops
    (the FP64 operation) against the measured sustained BF16 peak; the BF16
    slice-product flops they executed are reported beside, not in, the
    fraction.  The Cholesky products carry the captured DRAM bytes per tile
    scaled to a launch, as long as the kernel source is the captured one."""
    tiles = 1000.0
    n = 8192.0
    algo = n ** 3 / 3
    prof = {"chol_update": (10.0, 5, algo, tiles * bench.OZAKI_TILE_FLOPS), "sweep": (1.0, 1, 1.0, 1.0)}
    rf, cls = bench.roofline(prof, 1, "mixed")
    peaks, _src = bench.measured_peaks()
    assert cls == "chol_update" and rf["bound"] == "tensor"
    assert rf["peak"] == peaks["bf16_tflops_sustained"]
    assert rf["achieved"] == pytest.approx(algo / 0.010 / 1e12)
    assert rf["frac"] == pytest.approx(algo / 0.010 / 1e12 / rf["peak"])
    assert rf["executed_tflops"] == pytest.approx(tiles * bench.OZAKI_TILE_FLOPS / 0.010 / 1e12)
    if bench.ozaki_source_hash().startswith(bench.OZAKI_TRAFFIC["source_sha256_prefix"]):
        assert rf["traffic"] == pytest.approx(tiles * bench.OZAKI_TRAFFIC["bytes_per_tile"] / 5)
    else:
        assert rf["traffic"] is None


def test_headline_defaults_and_oracle_sample():
    """The default workload is the largest single-GPU configuration (24 x 24
    Heisenberg, Ns = 65536, CG), with the FP64 arm and the serving stream of
    512 requests; the oracle's bounded sample is a few chains of it."""
    import sys
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        a = bench.parse()
    finally:
        sys.argv = argv
    assert a.workload == "heis2d_24x24" and a.serve == 512 and not a.no_compare
    w = bench.workload(a.workload)
    assert (w["N"], w["M"], w["chains"] * w["per_chain"], w["solver"]) == (576, 4608, 65536, "cg")
    cfg = bench.workload_config(w, "mixed", 1)
    assert cfg["cg_tol"] == 1e-6 and bench.workload_config(w, "f64", 1)["cg_tol"] == 1e-10
    assert 1 <= bench.oracle_chains(a.workload) < w["chains"]
    assert bench.host_cores() >= 1


def test_l2_text_names_the_array_that_outgrows_l2():
    assert "larger" in bench.l2_text("cholesky_samplespace", 8192, 200, 20300)
    assert "SMALLER" in bench.l2_text("cholesky_samplespace", 1024, 200, 20300)
    assert "tanh(theta)" in bench.l2_text("cg", 16384, 1600, 642000)
    assert bench.replica_value(4, 10, 2000.0) == pytest.approx(20.0)


def test_jacobian_product_traffic_follows_the_captured_kernel(monkeypatch):
    """The CG products report the captured DRAM bytes of k_tc4 (the mean of a
    J v and a J^T g launch) scaled by the workload's samples, only while the
    kernel's source section is the one the capture was taken from."""
    prof = {"jvp_vjp": (100.0, 100, 3.49e13, 1e14), "sweep": (50.0, 8, 1e10, 1e10)}
    cap = bench.TC4_TRAFFIC
    monkeypatch.setattr(bench, "tc4_source_hash", lambda: cap["source_sha256_prefix"] + "0" * 48)
    rf, cls = bench.roofline(prof, 1, "mixed", ns=65536)
    assert cls == "jvp_vjp"
    assert rf["traffic"] == pytest.approx(0.5 * (cap["jv"] + cap["jtg"]) * 65536 / cap["ns"])
    rf_none, _ = bench.roofline(prof, 1, "mixed")  # no sample count: no scaled figure
    assert rf_none["traffic"] is None
    monkeypatch.setattr(bench, "tc4_source_hash", lambda: "f" * 64)  # the kernel has changed
    rf_stale, _ = bench.roofline(prof, 1, "mixed", ns=65536)
    assert rf_stale["traffic"] is None


def test_captured_sources_are_the_current_kernels():
    """The traffic constants belong to the kernels in the tree (a kernel
    change without a new capture turns the figure off, and this flags it)."""
    assert bench.tc4_source_hash().startswith(bench.TC4_TRAFFIC["source_sha256_prefix"])
    assert bench.ozaki_source_hash().startswith(bench.OZAKI_TRAFFIC["source_sha256_prefix"])
