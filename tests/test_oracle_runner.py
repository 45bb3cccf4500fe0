"""The multi-process whole-map oracle run equals the single-process oracle, and its accuracy gate
reproduces the parity tests' gate (CPU only)."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import pisco_oracle as O
from oracle import runner
from paper_2302_13431_gb300.phantoms import make_case


@pytest.fixture(scope="module")
def pool():
    p, w = runner.make_pool(3)
    yield p, w
    p.close()
    p.join()


def test_parallel_estimate_equals_single_process(pool):
    grid, Q, cs = (40, 48), 5, (18, 20)
    case = make_case(grid, Q, cs, seed=4, phase="poly4")
    ref = O.estimate(case.calib, grid, (2, 3), reduction=2, iters=30, seed=4, return_all=True, exact=False)
    par = runner.estimate_parallel(case.calib, grid, (2, 3), reduction=2, iters=30, seed=4, pool=pool[0],
                                   workers=pool[1])
    np.testing.assert_allclose(par["maps"], ref["maps"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(par["eig"], ref["eig"], rtol=0, atol=1e-12)
    assert par["k"] == ref["k"] and par["R"] == ref["R"]
    w = np.linalg.eigvalsh(ref["G"])[:, :2] / ref["lam"].shape[0]
    np.testing.assert_allclose(par["w2"], w, rtol=0, atol=1e-12)


def test_gate_masks_and_errors():
    grid, Q, cs = (40, 48), 5, (18, 20)
    case = make_case(grid, Q, cs, seed=5, phase="poly4")
    ref = runner.estimate_parallel(case.calib, grid, (2, 3), reduction=2, iters=30, seed=5, workers=2)
    full, red = runner.gate_masks(case.rho, ref["w2"], grid, 2)
    inner = ndimage.binary_erosion(np.abs(case.rho) > 0, iterations=2)
    assert not (full & ~inner).any() and red.shape == (20, 24)
    # a phase rotation per pixel is invisible to the measure; a perturbation is seen at its size
    ph = np.exp(1j * np.linspace(0, 6, int(np.prod(grid)))).reshape(grid)
    e0 = runner.gated_errors(ref["maps"] * ph[None], ref["eig"], ref, case.rho, 2)
    assert e0["map_err"] < 1e-12 and e0["eig_err"] == 0.0
    bad = ref["maps"].copy()
    bad[1] *= 1 + 1e-3
    e1 = runner.gated_errors(bad, ref["eig"] + 2e-5, ref, case.rho, 2)
    assert 1e-4 < e1["map_err"] < 1e-3 and abs(e1["eig_err"] - 2e-5) < 1e-12
