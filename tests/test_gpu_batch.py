"""Batched estimates (one CUDA graph, concurrent per-item branches) must equal the single-plan
path item by item, for items of different grid size, coil count and calibration size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoBatch, PiscoEstimator  # noqa: E402
from paper_2302_13431_gb300.phantoms import make_case  # noqa: E402

SPECS = [
    dict(grid=(64, 64), calib_shape=(24, 24), num_coils=8, tau=2, kernel_shape="rect", reduction=2, iters=20),
    dict(grid=(48, 40), calib_shape=(20, 18), num_coils=5, tau=(3, 2), reduction=2, iters=20),
    dict(grid=(96, 96), calib_shape=(24, 24), num_coils=16, tau=3, reduction=4, iters=20),
    dict(grid=(64, 64), calib_shape=(28, 28), num_coils=12, tau=3, reduction=4, iters=20),
    dict(grid=(16, 24, 20), calib_shape=(10, 12, 10), num_coils=4, tau=2, reduction=2, iters=20),
]


def _inputs():
    return [make_case(s["grid"], s["num_coils"], s["calib_shape"], seed=40 + i).calib
            for i, s in enumerate(SPECS)]


def test_batch_equals_single_plans_device_and_host():
    calibs_h = _inputs()
    calibs = [torch.from_numpy(c).cuda() for c in calibs_h]
    batch = PiscoBatch(SPECS)
    maps, eigs = batch.alloc_outputs()
    single_launches = 0
    for rep in range(3):  # eager, capture, replay
        batch.estimate_into(calibs, maps, eigs)
        torch.cuda.synchronize()
        assert all(s == B.PISCO_OK for s in batch.last_item_status), batch.last_item_status
        single_launches = 0
        for i, sp in enumerate(SPECS):
            est = PiscoEstimator(sp["grid"], sp["calib_shape"], sp["num_coils"], sp["tau"],
                                 kernel_shape=sp.get("kernel_shape", "ellipsoid"),
                                 reduction=sp["reduction"], iters=sp["iters"])
            m1, e1 = est(calibs[i])
            torch.cuda.synchronize()
            single_launches += est.stats()["launches"]
            assert torch.equal(m1, maps[i]), (rep, i)
            assert torch.equal(e1, eigs[i]), (rep, i)
            est.close()
    # host-buffer batch: same results
    hm = [np.empty(tuple(m.shape), np.complex64) for m in maps]
    he = [np.empty(tuple(e.shape), np.float32) for e in eigs]
    batch.estimate_host(calibs_h, hm, he)
    for i in range(len(SPECS)):
        np.testing.assert_array_equal(hm[i], maps[i].cpu().numpy())
        np.testing.assert_array_equal(he[i], eigs[i].cpu().numpy())
    info = batch.info()
    assert info["count"] == len(SPECS)
    # the last captured graph (host buffers) holds the single plans' kernels plus copies,
    # and only kernels count as launches
    assert info["launches"] == single_launches
    batch.close()


def test_batch_rejects_invalid_items():
    bad = dict(SPECS[0])
    bad["calib_shape"] = (4, 4)
    with pytest.raises(B.PiscoError):
        PiscoBatch([SPECS[0], bad])


def test_launch_and_wait_equal_the_blocking_host_call():
    calibs_h = _inputs()
    pin = lambda a: torch.from_numpy(a).pin_memory().numpy()  # noqa: E731
    cal = [pin(c) for c in calibs_h]
    a, b = PiscoBatch(SPECS), PiscoBatch(SPECS)
    ma = [pin(np.empty((s["num_coils"],) + tuple(s["grid"]), np.complex64)) for s in SPECS]
    mb = [pin(np.empty((s["num_coils"],) + tuple(s["grid"]), np.complex64)) for s in SPECS]
    ref = [np.empty((s["num_coils"],) + tuple(s["grid"]), np.complex64) for s in SPECS]
    a.estimate_host(calibs_h, ref)
    for step in range(4):  # ping-pong: two calls in flight
        (a if step % 2 == 0 else b).launch_host(cal, ma if step % 2 == 0 else mb)
        if step > 0:
            (b if step % 2 == 0 else a).wait()
    (b if 4 % 2 == 0 else a).wait()
    for i in range(len(SPECS)):
        np.testing.assert_array_equal(ma[i], ref[i])
        np.testing.assert_array_equal(mb[i], ref[i])
    a.launch_host(cal, ma)
    with pytest.raises(B.PiscoError):
        a.launch_host(cal, ma)  # one call in flight per batch object
    a.wait()
    with pytest.raises(B.PiscoError):
        a.wait()                # nothing launched
    a.close()
    b.close()


def test_device_launch_and_wait_in_turn_equal_the_blocking_call():
    """pisco_batch_launch / pisco_batch_wait on device buffers, two batch objects launched in turn
    on one stream with a stream write between steps: every step equals the blocking call."""
    dcal = [torch.from_numpy(c).cuda() for c in _inputs()]
    a, b = PiscoBatch(SPECS), PiscoBatch(SPECS)
    ref_m, ref_e = a.alloc_outputs()
    a.estimate_into(dcal, ref_m, ref_e)
    io = [a.alloc_outputs(), b.alloc_outputs()]
    scratch = torch.zeros(1 << 20, device="cuda")
    for step in range(5):
        scratch.add_(1.0)  # work on the caller's stream between steps
        (a, b)[step % 2].launch(dcal, *io[step % 2])
        if step > 0:
            (a, b)[(step - 1) % 2].wait()
    (a, b)[4 % 2].wait()
    torch.cuda.synchronize()
    for k in range(2):
        for i in range(len(SPECS)):
            assert torch.equal(io[k][0][i], ref_m[i]) and torch.equal(io[k][1][i], ref_e[i])
    assert float(scratch[0]) == 5.0
    a.launch(dcal, *io[0])
    with pytest.raises(B.PiscoError):
        a.launch(dcal, *io[0])  # one call in flight per batch object
    a.wait()
    a.close()
    b.close()
