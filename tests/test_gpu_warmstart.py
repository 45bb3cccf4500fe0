"""The learned warm start inside the estimate (pisco_set_warm_start).

* Path parity: with the network's proposals as start vectors, the GPU power iteration equals the
  FP64 oracle's power iteration from the oracle network's proposals on the same G(x).
* Gate: a gate that flags every pixel reproduces the plain path bitwise; no gate, no fallback.
* Gain: a patch network (3 x 3 neighbourhood of the normalised low-resolution vectors) trained by
  the library's kernels with the direction loss on pairs the method generates starts the power
  iteration far closer to the exact null vector than the method's own start, and closer than the
  heuristic y(x)/||y(x)|| it corrects, on held-out cases.
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import mlp_oracle as M
from oracle import pisco_oracle as O
from paper_2302_13431_gb300.phantoms import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoEstimator  # noqa: E402
from paper_2302_13431_gb300.warmstart import WarmStartNet, features, teacher_pairs  # noqa: E402

SMALL = dict(grid=(64, 64), Q=8, calib=(24, 24), tau=2, shape="rect", red=1)


def _est(cfg, iters=30, **kw):
    return PiscoEstimator(cfg["grid"], cfg["calib"], cfg["Q"], cfg["tau"], kernel_shape=cfg["shape"],
                          reduction=cfg["red"], iters=iters, **kw)


def test_warm_started_power_iteration_matches_oracle():
    cfg = SMALL
    Q = cfg["Q"]
    case = make_case(cfg["grid"], Q, cfg["calib"], seed=21, phase="linear")
    n_in = 9 * 2 * Q
    from paper_2302_13431_gb300.warmstart import he_init
    net = WarmStartNet(Q, 128, params=he_init(n_in, 128, 2 * Q, seed=4, last_scale=0.05), radius=1)
    est = _est(cfg)
    net.attach(est, iters=12, gate=0.0, fallback_iters=30)
    maps, eig = est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    assert est.stats()["warm_fallback"] == 0
    G = est.debug_buffer(B.PISCO_BUF_G).cpu().numpy().reshape(-1, Q, Q).astype(np.complex128)
    Y = est.debug_buffer(B.PISCO_BUF_Y).cpu().numpy().reshape(Q, -1).T.astype(np.complex128)
    V = est.debug_buffer(B.PISCO_BUF_V).cpu().numpy().reshape(Q, -1).T
    P = M.unpack(net.params(), n_in, 128, 2 * Q)
    out, _ = M.forward(P, M.patch_features(Y.T, cfg["grid"], 1))
    L = O.kernel_support((2, 2), "rect").shape[0]
    v, lam, _ = O.power_iteration(G, M.to_complex(out), 12, L)
    v = O.phase_align(v, Y)
    w = np.linalg.eigvalsh(G) / L
    inner = ndimage.binary_erosion(np.abs(case.rho) > 0, iterations=2).reshape(-1)
    sel = inner & ((w[:, 1] - w[:, 0]) > 1e-3)
    al = lambda a: a * np.exp(-1j * np.angle(a[:, :1]))  # noqa: E731
    err = np.linalg.norm((al(V) - al(v))[sel]) / np.linalg.norm(v[sel])
    assert err <= 1e-4, err
    assert np.abs(eig.cpu().numpy().reshape(-1) - lam)[sel].max() <= 1e-5
    net.close()
    est.close()


def test_gate_everywhere_equals_plain_path_and_no_gate_no_fallback():
    cfg = SMALL
    case = make_case(cfg["grid"], cfg["Q"], cfg["calib"], seed=22, phase="linear")
    calib = torch.from_numpy(case.calib).cuda()
    plain = _est(cfg)
    m0, e0 = plain(calib)
    net = WarmStartNet(cfg["Q"], 64, seed=5)
    est = _est(cfg)
    net.attach(est, iters=3, gate=1e-30, fallback_iters=30)
    for _ in range(3):  # eager, capture, replay
        m1, e1 = est(calib)
        torch.cuda.synchronize()
        assert torch.equal(m0, m1) and torch.equal(e0, e1)
        assert est.stats()["warm_fallback"] == cfg["grid"][0] * cfg["grid"][1]
    net.attach(est, iters=3, gate=0.0, fallback_iters=30)
    est(calib)
    assert est.stats()["warm_fallback"] == 0
    for e in (plain, est, net):
        e.close()


def _errors_vs_exact(G, v0s, L, iters_list):
    """Median of 1 - |v_t^H v*| (phase-free) after t FP64 power iterations, per start."""
    w, U = np.linalg.eigh(G)
    vstar = U[:, :, 0]
    out = {}
    for name, v0 in v0s.items():
        row = []
        for t in iters_list:
            v, _, _ = O.power_iteration(G, v0, t, L)
            row.append(float(np.median(1.0 - np.abs(np.sum(np.conj(v) * vstar, axis=1)))))
        out[name] = row
    return out


def test_trained_warm_start_beats_plain_and_heuristic_starts():
    """2D 96^2, Q = 8, 24^2 calibration, ellipse r = 3, f = 2: 200 training cases (about 110 k
    pairs), 20 validation cases, 3 held-out cases.  Measured on a GB300: the validation-selected
    network's median direction error on the held-out cases is 0.83x the heuristic's at the start
    and 0.49x after 5 iterations; the test asserts < 0.9x and < 0.75x."""
    cfg = dict(grid=(96, 96), Q=8, calib=(24, 24), tau=3, shape="ellipsoid", red=2)
    Q = cfg["Q"]
    R = 1  # 3 x 3 patch
    teacher, check = _est(cfg, iters=400), _est(cfg, iters=200)  # converged targets only
    ntr, nva = 200, 20
    X, T = teacher_pairs(teacher, [torch.from_numpy(make_case(cfg["grid"], Q, cfg["calib"], seed=300 + i).calib).cuda()
                                   for i in range(ntr)], eig_max=0.05, radius=R, check=check)
    Xv, Tv = teacher_pairs(teacher, [torch.from_numpy(make_case(cfg["grid"], Q, cfg["calib"], seed=300 + ntr + i)
                                                      .calib).cuda() for i in range(nva)], eig_max=0.05, radius=R,
                           check=check)
    net = WarmStartNet(Q, 128, seed=0, max_batch=8192, radius=R)
    n0 = min(8192, X.shape[0])
    loss0 = net.backward(X[:n0].contiguous(), T[:n0].contiguous())  # the untrained net = the heuristic
    hist = net.fit(X, T, epochs=6, batch=1024, lr=3e-4, seed=0, val=(Xv, Tv))
    loss1 = net.backward(X[:n0].contiguous(), T[:n0].contiguous())
    print(f"training loss per epoch {[f'{v:.2e}' for v in hist]}")
    print(f"training pairs {X.shape[0]}, loss {loss0:.5f} (heuristic) -> {loss1:.5f}; "
          f"validation direction error per epoch {[f'{v:.2e}' for v in net.val_history]}")
    assert min(net.val_history) <= net.val_history[0]
    L = O.kernel_support((3, 3), "ellipsoid").shape[0]
    iters_list = [0, 2, 5, 10, 20]
    agg = {}
    for s in range(3):  # held-out cases
        case = make_case(cfg["grid"], Q, cfg["calib"], seed=900 + s)  # held out
        est = _est(cfg)
        est(torch.from_numpy(case.calib).cuda())
        G = est.debug_buffer(B.PISCO_BUF_G).cpu().numpy().reshape(-1, Q, Q).astype(np.complex128)
        Y = est.debug_buffer(B.PISCO_BUF_Y).cpu().numpy().reshape(Q, -1).T.astype(np.complex128)
        eigv = np.linalg.eigvalsh(G) / L
        red = tuple(g // cfg["red"] for g in cfg["grid"])
        inner = ndimage.binary_erosion(np.abs(case.rho) > 0, iterations=2)[::cfg["red"], ::cfg["red"]].reshape(-1)
        sel = inner & ((eigv[:, 1] - eigv[:, 0]) > 1e-3)
        prop = net.forward(features(est, R)).cpu().numpy().astype(np.float64)
        starts = {"plain": O.start_vectors(0, red[0] * red[1], Q), "heuristic": Y, "learned": M.to_complex(prop)}
        e = _errors_vs_exact(G[sel], {k: v[sel] for k, v in starts.items()}, L, iters_list)
        for k, row in e.items():
            agg.setdefault(k, []).append(row)
        est.close()
    med = {k: np.median(np.array(v), axis=0) for k, v in agg.items()}
    for k, row in med.items():
        print(f"{k:9s} median 1-|<v_t,v*>| at t={iters_list}: " + " ".join(f"{x:.2e}" for x in row))
    # far closer than the method's own start, at every iteration count that is not yet converged
    assert med["learned"][0] < 1e-2 * med["plain"][0]
    assert med["learned"][1] < 1e-2 * med["plain"][1] and med["learned"][2] < 1e-2 * med["plain"][2]
    # the network corrects the heuristic start: closer to the null vector on unseen data, and the
    # gap widens over the first iterations (the correction removes slowly decaying components)
    ratio = med["learned"][0] / med["heuristic"][0]
    ratio5 = med["learned"][2] / med["heuristic"][2]
    print(f"learned / heuristic median direction error at t=0: {ratio:.3f}, after 5 iterations: {ratio5:.3f}")
    assert ratio < 0.9 and ratio5 < 0.75
    net.close()
    teacher.close()
    check.close()
