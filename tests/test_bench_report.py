"""The bench's roofline bookkeeping on CPU: algorithmic bytes per kernel and launch, the
bound chosen per form, the explicit variant's words, and the traffic lookup keyed by the
kernel-source hash."""
import math

import bench


class _Case:
    nx, ny = 512, 256


def test_fp32_line_reports_hbm_fractions_from_words():
    cells = 6 * 512 * 256
    ktot = {"predict": 2.0, "correct": 1.0, "fill_C": 0.5}   # ms over 100 steps
    kcount = {"predict": 100, "correct": 100, "fill_C": 100}
    r = bench.roofline(ktot, kcount, 100, cells, 4, _Case, 6000.0, "measured", "fp32")
    assert r["bound"] == "hbm" and r["kernel"] == "predict"
    alg = bench.KERNEL_STEP_WORDS["predict"][0] * 4 * cells
    assert math.isclose(r["alg_bytes_per_launch"], alg)
    assert math.isclose(r["achieved"], alg / 20e-6 / 1e9)
    assert math.isclose(r["frac"], r["achieved"] / 6000.0)
    assert r["kernels"]["fill_C"].get("hbm_frac") is None          # ghost kernels: no words
    assert math.isclose(r["kernels"]["correct"]["hbm_frac"],     # table values are rounded
                        bench.KERNEL_STEP_WORDS["correct"][0] * 4 * cells / 10e-6 / 1e9 / 6000.0,
                        rel_tol=1e-3)


def test_fp64_2d_line_is_alu_bound_and_3d_is_hbm():
    cells = 6 * 512 * 256
    r = bench.roofline({"predict": 30.0}, {"predict": 100}, 100, cells, 8, _Case, 6000.0, "measured", "fp64")
    assert r["bound"] == "alu" and r["unit"].startswith("GFLOP")
    flops = bench.kernel_flops64("predict", 512, 256) * cells
    assert math.isclose(r["achieved"], flops / 300e-6 / 1e9)
    r3 = bench.roofline({"predict": 30.0}, {"predict": 100}, 100, cells, 8, _Case, 6000.0, "measured",
                        "fp64", bench.KERNEL_STEP_WORDS_3D)
    assert r3["bound"] == "hbm"


def test_explicit_words_halve_the_single_solve():
    w = bench.explicit_words(bench.KERNEL_STEP_WORDS_3D, ("rows_fwd", "y_fft", "z_solve", "y_ifft"))
    for k in ("rows_fwd", "y_fft", "z_solve", "y_ifft"):
        assert w[k][0] * 2 == bench.KERNEL_STEP_WORDS_3D[k][0]
    assert w["rows_inv"] == (4, 4, 0)
    assert w["predict"] == bench.KERNEL_STEP_WORDS_3D["predict"]
    w2 = bench.explicit_words(bench.KERNEL_STEP_WORDS, ("rows_fwd", "cols_solve"))
    # a 2D FP64 line with the explicit words is still reported against the FP64 pipe
    r = bench.roofline({"predict": 30.0}, {"predict": 100}, 100, 1000, 8, _Case, 6000.0, "m", "fp64", w2)
    assert r["bound"] == "alu"


def test_traffic_lookup_requires_matching_kernel_sources(tmp_path, monkeypatch):
    sha = bench.kernel_sources_sha()
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_w_fp32.txt").write_text(
        f"kernel=predict dram_bytes_per_launch=123 csrc_sha={sha}\n"
        "kernel=correct dram_bytes_per_launch=456 csrc_sha=0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "kernel_sources_sha", lambda: sha)
    assert bench.read_traffic("predict", "fp32", "w") == 123.0
    assert bench.read_traffic("correct", "fp32", "w") is None     # taken on other sources
    assert bench.read_traffic("predict", "fp64", "w") is None     # no capture


def test_tensor_core_solve_reports_its_tensor_rate():
    # 256^3: 2 x 256 rows x 130 padded complex columns of the half spectrum = 66560 real
    # columns; each takes, forward and inverse, 2 products of a 128 x 128 matrix (after the
    # even/odd step) in 3 split parts: 66560 x 2 x 2 x 3 x 2 x 128^2 flops
    flops = bench.tc_zsolve_flops(256, 256, 256)
    assert flops == 66560 * 2 * 2 * 3 * 2 * 128 * 128
    assert bench.tc_zsolve_flops(128, 128, 128) == (2 * 128 * 66) * 2 * 1 * 3 * 2 * 128 * 128

    class C3:
        nx = ny = nz = 256

    cells = 256 ** 3
    ktot = {"predict": 3.0, "z_solve_tc": 1.0}          # ms over 10 steps, 2 launches per step
    kcount = {"predict": 10, "z_solve_tc": 20}
    r = bench.roofline(ktot, kcount, 10, cells, 4, C3, 6000.0, "measured", "fp32_3xbf16",
                       bench.KERNEL_STEP_WORDS_3D, workload="sphere_256", dim=3)
    e = r["kernels"]["z_solve_tc"]
    tp, _ = bench.measured_bf16_peak()
    assert math.isclose(e["tensor_TFLOPs"], round(flops * 20 / 1e-3 / 1e12, 1), rel_tol=1e-9)
    assert math.isclose(e["tensor_frac"], round(flops * 20 / 1e-3 / 1e12 / tp, 4), rel_tol=1e-9)
    assert "hbm_frac" in e                                # the same words as the FFT solve
