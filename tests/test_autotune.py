"""Autotuner: candidates stay within the FP32 parity gates; on a GPU the chosen configuration is
the fastest of its table, is cached, and the tuned batch still matches the single plans."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2302_13431_gb300.autotune import KNOB_KEYS, candidates  # noqa: E402


def test_candidates_exclude_single_pass_routes():
    cs = candidates()
    assert len(cs) == len({tuple(sorted(c.items())) for c in cs})
    assert all(set(c) == set(KNOB_KEYS) for c in cs)
    assert all("1pass" not in c["precision"] for c in cs)
    assert {c["precision"] for c in cs} == {"fp32", "tc_g", "tc_g_eig", "tc_all"}


@pytest.mark.gpu
def test_tune_picks_the_fastest_and_caches(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2302_13431_gb300 import _binding as B
    from paper_2302_13431_gb300.autotune import apply, tune
    from paper_2302_13431_gb300.estimator import PiscoBatch, PiscoEstimator
    from paper_2302_13431_gb300.phantoms import make_case
    specs = [dict(grid=(64, 64), calib_shape=(24, 24), num_coils=8, tau=3, reduction=2, iters=20)] * 3
    cache = str(tmp_path / "tune.json")
    cands = [dict(precision="fp32", tc_splits=0, gemm_splits=0, gemm_tile=0, gram_df=False, tc_interp=False,
                  batch_group=0),
             dict(precision="tc_g_eig", tc_splits=4, gemm_splits=2, gemm_tile=64, gram_df=True, tc_interp=True,
                  batch_group=0)]
    cfg, table = tune(specs, steps=2, warmup=2, cache=cache, cands=cands)
    assert all(r["ms"] is not None for r in table), table  # both candidates pass the correctness gate
    assert cfg == {k: min(table, key=lambda r: r["ms"])[k] for k in KNOB_KEYS}
    cfg2, table2 = tune(specs, cache=cache, cands=cands)  # cached: no re-timing
    assert cfg2 == cfg and table2 == table
    calibs = [torch.from_numpy(make_case((64, 64), 8, (24, 24), seed=70 + i).calib).cuda() for i in range(3)]
    b = PiscoBatch(apply(specs, cfg))
    maps, eigs = b.alloc_outputs()
    b.estimate_into(calibs, maps, eigs)
    for i in range(3):
        est = PiscoEstimator((64, 64), (24, 24), 8, 3, reduction=2, iters=20, precision=cfg["precision"],
                             tc_splits=cfg["tc_splits"], gemm_splits=cfg["gemm_splits"], gemm_tile=cfg["gemm_tile"],
                             gram_df=cfg["gram_df"], tc_interp=cfg["tc_interp"])
        m1, e1 = est(calibs[i])
        torch.cuda.synchronize()
        assert torch.equal(m1, maps[i]) and torch.equal(e1, eigs[i])
        est.close()
    b.close()
    assert B.PISCO_OK == 0
