"""bench.py's roofline arithmetic on the CPU: the algorithmic bytes and flops
of the i pass follow from the grid size and the transformed planes, and the
entry reports the resource the kernel is closer to (HBM or the float32
pipes) with the other fraction beside it."""
import math

import pytest

import bench


def test_i_pass_model_counts_the_transformed_planes():
    n, npl, nb = 128, 32, 64
    nbytes, flops = bench.kernel_model(n, 4, 1000, npl, nb)["conv_i"]
    B = 2 * npl * n * n * 8                       # float32 complex rows after the j pass
    assert nbytes == pytest.approx(2 * B + (n + 1) ** 3 * 4 / nb)
    L = 2 * n
    assert flops == pytest.approx(2 * (2 * n * n) * 5 * L * math.log2(L) + 2 * (2 * n * n) * L)


def test_roofline_reports_the_binding_resource():
    n, npl, nb, hbm = 128, 32, 64, 6662.6
    nbytes, flops = bench.kernel_model(n, 4, 1000, npl, nb)["conv_i"]
    # a launch time at which the float32 pipes are the closer bound
    t_ms = 0.922
    r = bench.roofline_for("conv_i.f32", t_ms * 40, 40, n, 1000, hbm, "measured", npl, nb)
    a_alu = flops * nb / (t_ms / 1000) / 1e12
    a_hbm = nbytes * nb / (t_ms / 1000) / 1e9
    assert r["bound"] == "alu"
    assert r["frac"] == pytest.approx(a_alu / (2 * bench.FP32_LANE_PEAK_T))
    assert r["frac_hbm"] == pytest.approx(a_hbm / hbm)
    assert r["frac"] > r["frac_hbm"]
    tr = bench.NCU_TRAFFIC[("conv_i.f32", 128, 64)]
    assert r["traffic"] == tr and r["traffic_GBps"] == pytest.approx(tr / (t_ms / 1000) / 1e9)
    # the same bytes with far fewer flops per byte: HBM is the bound
    r2 = bench.roofline_for("conv_jfwd.f32", 0.18 * 40, 40, n, 1000, hbm, "measured", npl, nb)
    assert r2["bound"] == "hbm" and r2["frac"] == pytest.approx(r2["frac_hbm"])
    assert r2["unit"] == "GB/s"


def test_fp32_peak_from_unit_counts():
    # 152 SMs x 128 float32 lanes x 2.07 GHz, in T lane operations per second
    assert bench.FP32_LANE_PEAK_T == pytest.approx(40.27, rel=1e-3)
