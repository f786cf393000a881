"""The bench line's roofline objects from per-kernel timings (host logic,
no GPU): the dominant kernel is the one with the most time, its bound the
resource it comes closer to (FP64 arithmetic against the derived FP64 peak,
or bytes against the measured copy bandwidth), frac = achieved / peak, the
traffic estimate scaled from the capture's DRAM-to-algorithmic ratio, and
the shares summing to one."""
import math

import bench


def timings():
    # (ms, launches, algorithmic bytes, FP64 flops) over the timed steps
    return {"sweep": (60.0, 60, 60 * 6.67e9, 60 * 1.9e7),
            "spmv": (64.0, 60, 60 * 6.74e9, 60 * 1.12e9),
            "mdot": (24.0, 60, 60 * 1.15e9, 60 * 1.1e7),
            "inverse": (174.0, 4, 16.0 * 7.9e8, 2.0 * 7.2e10)}


def test_dominant_kernel_and_bound():
    hbm = 6702.2
    k = bench._kernels_from_timing(timings(), hbm)
    assert math.isclose(sum(v["share"] for v in k.values()), 1.0)
    top = max(k, key=lambda n: k[n]["ms"])
    assert top == "inverse"
    r = bench._roofline_of(top, k[top], hbm, "measured", "stokes3d")
    assert r["bound"] == "alu" and r["peak"] == bench.FP64_PEAK_TFLOPS
    assert math.isclose(r["achieved"], 2.0 * 7.2e10 / 0.174 / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / r["peak"])
    assert 0.0 < r["frac"] < 1.0
    tr = bench.TRAFFIC[("stokes3d", "inverse")]["ratio"]
    assert math.isclose(r["traffic"], tr * k[top]["alg_bytes_per_launch"])
    s = bench._roofline_of("sweep", k["sweep"], hbm, "measured", "stokes3d")
    assert s["bound"] == "hbm" and s["unit"] == "GB/s"
    assert math.isclose(s["achieved"], 6.67e9 / 1e-3 / 1e9)
    assert math.isclose(s["frac"], s["achieved"] / hbm)


def test_no_traffic_without_a_capture():
    k = bench._kernels_from_timing(timings(), 6702.2)
    r = bench._roofline_of("mdot", k["mdot"], 6702.2, "measured", "diffusion3d")
    assert r["traffic"] is None and r["traffic_source"] is None


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2 FP64 FMA per clock x 2 flops x 2.07 GHz
    assert math.isclose(bench.FP64_PEAK_TFLOPS, 152 * 2 * 2 * 2.07e9 / 1e12)
