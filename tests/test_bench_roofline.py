"""bench.py's roofline bookkeeping on CPU: every operation name the plan's profiler can report
yields a roofline record, and the work formulas agree with the operation counts written out
independently here (complex multiply-add = 8 real flops)."""
import math
import os
import re
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402

W = bench.WORKLOAD
STATS = {"filter_len": 29, "eig_block": 64, "jacobi_sweeps": 4, "eig_iters": 6}
PEAKS = {"hbm_gbs": 6784.2, "bf16_tflops": 1868.0}


def _op_names():
    src = open(os.path.join(os.path.dirname(bench.__file__), "paper_2302_13431_gb300", "csrc", "pisco_api.cu")).read()
    return sorted(set(re.findall(r'OP\("([A-Za-z0-9_]+)"', src)))


def test_every_profiled_op_has_a_record():
    names = _op_names()
    assert "eig_gemm_AX" in names and "g_field_sep" in names and "gram_pairs_df" in names
    for op in names:
        prof = {op: (2.0, 40), "gram_pairs_df": (1.0, 20)}
        for prec in ("fp32", "tc_g_eig"):
            for ti in (False, True):
                r = bench.roofline_for(op, prof, W, STATS, PEAKS, prec, ti, 20)
                assert r["bound"] in ("alu", "tensor", "hbm", "latency")
                if r["achieved"] is not None:
                    assert math.isfinite(r["achieved"]) and r["achieved"] > 0 and r["peak"] > 0


def _ellipse_points(t):
    return [(y, x) for y in range(-t, t + 1) for x in range(-t, t + 1) if y * y + x * x <= t * t]


def test_lag_count_of_the_radius_3_ellipse():
    pts = _ellipse_points(3)
    assert len(pts) == 29 == STATS["filter_len"]
    diffs = {(a[0] - b[0], a[1] - b[1]) for a in pts for b in pts}
    assert bench.n_lags(W) == len(diffs)


@pytest.mark.parametrize("op, flops_per_map", [
    # two separable passes per coil pair: lags -> (rows x columns of x2), rows -> pixels
    ("g_field_sep", lambda Q, nl, nr1, nr2, B, n, m, L, Bg: 8 * Q * Q * (nl * nr2 + B * nr1 * nr2)),
    # P = U diag(w) U^H, one n x n x m product per map
    ("g_herk_tc", lambda Q, nl, nr1, nr2, B, n, m, L, Bg: 8 * n * n * m),
    # the orthogonal iteration's A X products plus the Rayleigh-Ritz one
    ("eig_gemm_AX", lambda Q, nl, nr1, nr2, B, n, m, L, Bg: 8 * n * n * m * (STATS["eig_iters"] + 1)),
])
def test_per_map_work_over_per_map_time(op, flops_per_map):
    Q = W["Q"]
    nr1, nr2 = W["grid"][0] // W["reduction"], W["grid"][1] // W["reduction"]
    B = 4 * W["tau"] + 1
    n, m = Q * STATS["filter_len"], STATS["eig_block"]
    L = W["calib"][0] + 2 * W["tau"]
    nmaps, ms_per_map = 20, 0.05
    prof = {op: (ms_per_map * nmaps, 7 * nmaps)}  # several profiled calls per map
    r = bench.roofline_for(op, prof, W, STATS, PEAKS, "tc_g_eig", True, nmaps)
    want = flops_per_map(Q, bench.n_lags(W), nr1, nr2, B, n, m, L, B) / (ms_per_map * 1e-3) / 1e12
    assert r["achieved"] == pytest.approx(want, rel=1e-12)


def test_fused_gram_pair_stage_counts():
    Q, t = W["Q"], W["tau"]
    L, B = W["calib"][0] + 2 * t, 4 * t + 1
    npair = Q * (Q + 1) // 2
    # per pair: the frequency-domain product (double-float, 60 FP32 instructions per complex
    # multiply-add), the contiguous-axis and axis-1 passes (Dot2 sums; the lags +d and -d share
    # their cosine and sine sums, 24 per complex term and lag), against the FP32 issue rate
    inst = npair * (60 * L * L + 24 * (L * L * B + B * B * L))
    prof = {"gram_pairs_df": (1.0, 20)}
    r = bench.roofline_for("gram_pairs_df", prof, W, STATS, PEAKS, "tc_g_eig", True, 20)
    assert r["achieved"] == pytest.approx(inst / 0.05e-3 / 1e12, rel=1e-12)
    assert r["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12, rel=1e-12) and r["unit"] == "Tinst/s"
    # with the fused stage present, the forward DFT record counts the forward passes only (one
    # launch per coil set does both of them)
    nc = W["calib"][0]
    prof = {"gram_dft_df": (1.0, 20), "gram_pairs_df": (1.0, 20)}
    r = bench.roofline_for("gram_dft_df", prof, W, STATS, PEAKS, "tc_g_eig", True, 20)
    fwd = Q * nc * L * nc + Q * L * L * nc
    assert r["achieved"] == pytest.approx(60 * fwd / 0.05e-3 / 1e12, rel=1e-12)
    # a launch over 8 map sets does 8 times the work
    r8 = bench.roofline_for("gram_pairs_df", {"gram_pairs_df": (1.0, 20)}, W, STATS, PEAKS, "tc_g_eig", True, 160, 8)
    assert r8["achieved"] == pytest.approx(8 * inst / 0.05e-3 / 1e12, rel=1e-12)
