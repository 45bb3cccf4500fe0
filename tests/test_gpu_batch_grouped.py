"""Batched passes over items of identical parameters (every stage one launch over all items of a
group) must give, item by item, exactly the single-plan result: the same kernels run per item
with the same split decisions, so maps and eigenvalues are bitwise equal.  Covered: the routes the
autotuner may pick (2D and 3D), the grid-reduction-free path, host buffers, groups split by
batch_group, and items re-run alone through their views (eigensolver block saturated)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoBatch, PiscoEstimator  # noqa: E402
from paper_2302_13431_gb300.phantoms import make_case  # noqa: E402

BASE_2D = dict(grid=(96, 96), calib_shape=(24, 24), num_coils=12, tau=3, reduction=4, iters=20)
ROUTES = {
    "tuned": dict(precision="tc_g_eig", tc_splits=1, gemm_splits=2, gemm_tile=64, gram_df=True, tc_interp=True),
    "tc_all_split": dict(precision="tc_all", tc_splits=4, gram_df=True),
    "tc_g_fp64gram": dict(precision="tc_g", gemm_splits=2, gemm_tile=64),
    "tc_g_eig_auto": dict(precision="tc_g_eig"),
}


def _single(sp, calib, host=False):
    est = PiscoEstimator(sp["grid"], sp["calib_shape"], sp["num_coils"], sp["tau"],
                         kernel_shape=sp.get("kernel_shape", "ellipsoid"), reduction=sp["reduction"],
                         iters=sp["iters"], precision=sp.get("precision", "fp32"), tc_splits=sp.get("tc_splits", 0),
                         gemm_splits=sp.get("gemm_splits", 0), gemm_tile=sp.get("gemm_tile", 0),
                         gram_df=sp.get("gram_df", False), tc_interp=sp.get("tc_interp", False),
                         eig_block=sp.get("eig_block", 0))
    m1, e1 = est(calib)
    torch.cuda.synchronize()
    st, stats = est.last_status, est.stats()
    est.close()
    return m1, e1, st, stats


def _check_batch(specs, seeds, reps=3):
    calibs = [torch.from_numpy(make_case(sp["grid"], sp["num_coils"], sp["calib_shape"], seed=s).calib).cuda()
              for sp, s in zip(specs, seeds)]
    batch = PiscoBatch(specs)
    maps, eigs = batch.alloc_outputs()
    ref = [_single(sp, c) for sp, c in zip(specs, calibs)]
    for rep in range(reps):  # eager, capture, replay
        batch.estimate_into(calibs, maps, eigs)
        torch.cuda.synchronize()
        for i, (m1, e1, st, stats) in enumerate(ref):
            assert batch.last_item_status[i] == st == B.PISCO_OK, (rep, i, batch.last_item_status[i], st)
            assert torch.equal(m1, maps[i]), (rep, i)
            assert torch.equal(e1, eigs[i]), (rep, i)
            assert batch.item_stats(i)["signal_dim"] == stats["signal_dim"], (rep, i)
    return batch, calibs, maps, eigs


@pytest.mark.parametrize("route", sorted(ROUTES))
def test_grouped_batch_equals_single_plans(route):
    specs = [dict(BASE_2D, **ROUTES[route])] * 5
    batch, _, _, _ = _check_batch(specs, [300 + i for i in range(5)])
    info = batch.info()
    # one group: far fewer launches than five chains of a single plan each
    assert info["launches"] > 0
    batch.close()


def test_grouped_batch_3d_dense_G_and_no_reduction():
    tuned = ROUTES["tuned"]
    specs3 = [dict(grid=(16, 24, 20), calib_shape=(10, 12, 10), num_coils=4, tau=2, reduction=2, iters=20,
                   **tuned)] * 3
    _check_batch(specs3, [400, 401, 402])[0].close()
    specs_f1 = [dict(grid=(48, 48), calib_shape=(20, 20), num_coils=6, tau=2, kernel_shape="rect", reduction=1,
                     iters=20, precision="tc_g_eig", gram_df=True)] * 4
    _check_batch(specs_f1, [410, 411, 412, 413])[0].close()


def test_batch_group_splits_and_mixed_shapes():
    """batch_group=2 over five identical items (groups 2 + 2 + 1) plus two items of other shapes."""
    tuned = dict(ROUTES["tuned"], batch_group=2)
    other = dict(grid=(64, 64), calib_shape=(20, 20), num_coils=8, tau=2, reduction=2, iters=20, **ROUTES["tuned"])
    specs = [dict(BASE_2D, **tuned)] * 5 + [other, dict(other, num_coils=9)]
    _check_batch(specs, [500 + i for i in range(7)])[0].close()


def test_saturated_items_rerun_alone_through_their_views():
    """A block of 8 columns is too small for these data: every item saturates, is re-run alone with
    a doubled block (as a single plan is), and its group adopts the block for later calls."""
    specs = [dict(BASE_2D, eig_block=8, **ROUTES["tuned"])] * 3
    batch, calibs, maps, eigs = _check_batch(specs, [600, 601, 602])
    assert all(batch.item_stats(i)["eig_block"] > 8 for i in range(3))
    batch.close()


def test_grouped_batch_host_buffers_and_two_in_flight():
    """Host-buffer calls of a grouped batch, and two grouped batch objects launched in turn with
    different inputs every step: every output equals the single-plan result of its own input."""
    specs = [dict(BASE_2D, **ROUTES["tuned"])] * 4
    cases = [[make_case(BASE_2D["grid"], BASE_2D["num_coils"], BASE_2D["calib_shape"], seed=700 + 10 * s + i).calib
              for i in range(4)] for s in range(4)]
    refs = [[_single(specs[0], torch.from_numpy(c).cuda()) for c in step] for step in cases]
    pair = (PiscoBatch(specs), PiscoBatch(specs))
    pins = [[torch.from_numpy(c).pin_memory().numpy() for c in step] for step in cases]
    outs = [([torch.empty((12, 96, 96), dtype=torch.complex64).pin_memory().numpy() for _ in range(4)],
             [torch.empty((24, 24), dtype=torch.float32).pin_memory().numpy() for _ in range(4)]) for _ in range(2)]
    for rnd in range(2):  # the first round runs eagerly / captures, the second replays
        for s in range(4):
            pair[s % 2].launch_host(pins[s], *outs[s % 2])
            if s > 0:
                pair[(s - 1) % 2].wait()
                prev = s - 1
                for i in range(4):
                    np.testing.assert_array_equal(outs[prev % 2][0][i], refs[prev][i][0].cpu().numpy())
                    np.testing.assert_array_equal(outs[prev % 2][1][i], refs[prev][i][1].cpu().numpy())
        pair[3 % 2].wait()
        for i in range(4):
            np.testing.assert_array_equal(outs[1][0][i], refs[3][i][0].cpu().numpy())
    for b in pair:
        b.close()
