"""Host-side logic of bench.py that needs no GPU: workload defaults and the
kernel-family table the roofline line is built from."""
import bench


def test_workload_sizes_default_per_configuration():
    assert bench.parse([]).n == 100000
    assert bench.parse(["--workload", "band4"]).n == 100000
    assert bench.parse(["--workload", "band16"]).n == 32768
    assert bench.parse(["--workload", "band16", "--n", "4096"]).n == 4096
    a = bench.parse([])
    assert a.leaf == 256 and a.tol == 1e-10 and a.warmup >= 3 and a.tsqr_chunk == 0 and not a.autotune


def test_kernel_table_groups_gemm_call_sites_and_orders_by_time():
    prof = {
        "k_gemm": (10, 2.0, 2.0e9),
        "k_gemm[chol]": (30, 3.0, 1.0e9),
        "k_gemm[mult]": (5, 5.0, 4.0e9),
        "k_gemm_tc": (4, 1.0, 1.0e9),
        "k_qr": (7, 4.0, 1.6e9),
        "k_givens": (1, 9.0, 0.0),
        "host_wait": (100, 50.0, 0.0),
        "k_unused": (0, 0.0, 0.0),
    }
    t = bench.kernel_table(prof, givens_rotations=3 * 1000 - 2)
    # call-site buckets of the binary64 GEMM form one family; the tensor-core
    # GEMM and host waits are not folded in; empty families are dropped
    assert t["k_gemm"]["launches"] == 45 and abs(t["k_gemm"]["ms"] - 10.0) < 1e-12
    assert abs(t["k_gemm"]["gflop"] - 7.0) < 1e-9
    assert "host_wait" not in t and "k_unused" not in t and "k_gemm_tc" in t
    # ordered by time; TFLOP/s = flops / time; fraction of the binary64 rate
    assert list(t)[0] == "k_gemm"
    assert abs(t["k_gemm"]["tflops"] - 7.0e9 / 10.0e-3 / 1e12) < 1e-3
    assert abs(t["k_gemm"]["frac_fp64"] - t["k_gemm"]["tflops"] / bench.FP64_PEAK_TFLOPS) < 1e-3
    # the Givens chain reports its critical path per rotation instead of a rate
    assert abs(t["k_givens"]["ns_per_rotation"] - 9.0e6 / 2998) < 0.1
    assert "frac_fp64" not in t["k_givens"]
    assert abs(sum(v["share"] for v in t.values()) - 1.0) < 1e-3
