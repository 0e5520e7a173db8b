"""bench.py's cost model and roofline arithmetic on the host (no device): the per-tau
algorithmic work of the dense and virtual-space routes, the tensor-product factors of the
two precisions, and the per-stage table the bench prints."""
import math

import bench


SIZES = {"n_pw": 3071, "n_occ": 32, "grid": 24}


def _costs(nv, wv, green_full=False, reps=1):
    return bench.stage_costs(SIZES, 836, True, reps, 15, nv, wv, 3039, green_full)


def test_stage_costs_count_each_route():
    dense = _costs([3039], [0])
    virt = _costs([100], [1])
    ncols = 836 * 32
    assert math.isclose(dense["w_gemm"]["flops"], 4.0 * ncols * 3071 * 3071)
    assert math.isclose(dense["green_gemm"]["flops"], 2.0 * 3071 * 3071 * 3039)
    # through the virtual space: two products over the kept virtuals, no Green's function
    assert math.isclose(virt["w_gemm"]["flops"], 4.0 * ncols * 3071 * 2 * 100)
    assert virt["green_gemm"]["flops"] == 0.0
    # the Green's function on the tensor cores sums over every virtual
    assert math.isclose(_costs([100], [0], green_full=True)["green_gemm"]["flops"], 2.0 * 3071 * 3071 * 3039)
    assert math.isclose(_costs([3039, 100], [0, 1], reps=2)["w_gemm"]["flops"],
                        2 * (dense["w_gemm"]["flops"] + virt["w_gemm"]["flops"]))
    line = 5.0 * 24 * math.log2(24)
    assert math.isclose(dense["plane_fft"]["flops"], ncols * 32 * 24 * (24 + 15) * line)


def test_stage_rooflines_use_each_stage_bound():
    st = {"w_gemm": {"ms": 100.0, "launches": 10}, "plane_fft": {"ms": 400.0, "launches": 8},
          "accumulate": {"ms": 1.0, "launches": 8}, "idle": {"ms": 0.0, "launches": 0}}
    costs = _costs([3039], [0])
    peaks = {"hbm_gbs": 6760.6, "bf16_tflops": 1905.5}
    alu = {"fp64": 1.2, "fp32": 73.0, "kind": "test"}
    for precision, factor in ((0, 36.0), (1, 3.0)):
        r = bench.stage_rooflines(st, costs, precision, False, peaks, "measured", alu)
        assert set(r) == {"w_gemm", "plane_fft", "accumulate"}
        w = r["w_gemm"]
        assert w["bound"] == "tensor" and math.isclose(w["work_per_launch"], costs["w_gemm"]["flops"] / 10 * factor)
        assert math.isclose(w["achieved"], w["work_per_launch"] / 10e-3 / 1e12)
        assert math.isclose(w["peak"], 1905.5 * bench.TF32_OVER_BF16)
        p = r["plane_fft"]
        assert p["bound"] == "alu" and p["peak"] == (alu["fp64"] if precision == 0 else alu["fp32"])
        assert "bound" not in r["accumulate"] and math.isclose(r["accumulate"]["avg_launch_ms"], 1.0 / 8)
        dom = bench.roofline_of(st, costs, precision, False, peaks, "measured", alu)
        assert dom["kernel"] == "plane_fft" and math.isclose(dom["frac"], p["frac"])
    # CUDA-core GEMMs: the FP64 FMA rate bounds the product
    r = bench.stage_rooflines(st, costs, 0, True, peaks, "measured", alu)
    assert r["w_gemm"]["bound"] == "alu" and r["w_gemm"]["peak"] == alu["fp64"]


def test_stored_traffic_is_keyed_by_the_kernel_sources():
    for stage in bench.STAGE_SOURCES:
        assert len(bench.source_sha(stage)) == 16
    for precision in (0, 1):
        t = bench.traffic_for("plane_fft", precision)
        assert t is None or t > 0
    assert bench.traffic_for("accumulate", 0) is None
