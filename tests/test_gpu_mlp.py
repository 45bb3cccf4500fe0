"""The warm-start network's CUDA kernels (through the C ABI; tensor-core products with FP16
operands) against the FP64 oracle MLP: forward pass, both losses, every gradient, one Adam
step, the patch features; determinism of the batch reductions.

Tolerances: the oracle rounds the same operands to FP16 (weights, inputs, activations,
per-sample gradients), so the bulk agrees to FP32 accumulation (<= 2e-6 relative at the
median).  An activation within an FP32 rounding of an FP16 rounding boundary may round the
other way on one side: such isolated flips move an output by at most a few FP16 ulps of one
term (max error <= 2e-3 relative); the gradients, sums over the batch, stay within
1e-4 sqrt(B/256) of max|g|."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.warmstart import WarmStartNet, he_init  # noqa: E402


def _close(out, ref):
    scale = max(1.0, np.abs(ref).max())
    d = np.abs(out - ref).reshape(-1) / scale
    assert np.median(d) <= 2e-6 and d.max() <= 2e-3, (np.median(d), d.max())


@pytest.mark.parametrize("n_io,H,B,radius,loss", [(16, 128, 700, 0, "mse"), (64, 128, 4096, 0, "mse"),
                                                  (10, 37, 129, 0, "mse"), (16, 128, 3000, 1, "direction"),
                                                  (16, 64, 5000, 1, "mse"), (64, 128, 2500, 0, "direction")])
def test_forward_loss_and_gradients_match_oracle(n_io, H, B, radius, loss):
    rng = np.random.default_rng(n_io + H + B)
    n_in = (2 * radius + 1) ** 2 * n_io
    p = he_init(n_in, H, n_io, seed=n_io)
    p = p + (rng.standard_normal(p.size) * 0.05).astype(np.float32)
    net = WarmStartNet(n_io // 2, H, params=p, max_batch=8192, radius=radius, loss=loss)
    x = rng.standard_normal((B, n_in)).astype(np.float32)
    t = rng.standard_normal((B, n_io)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = net.forward(xd).cpu().numpy()
    P = M.unpack(p, n_in, H, n_io)
    ref, _ = M.forward(P, x)
    _close(out, ref)
    kind = 1 if loss == "direction" else 0
    lv = net.backward(xd, td)
    L, g = M.backward(P, x, t, kind=kind)
    assert abs(lv - L) <= 1e-4 * L
    gg = M.unpack(net.grads(), n_in, H, n_io)
    tol = 1e-4 * max(1.0, np.sqrt(B / 256))  # FP32 sums over the batch, fixed order
    for k in M.LAYERS:
        err = np.abs(gg[k] - g[k]).max() / max(np.abs(g[k]).max(), 1e-12)
        assert err <= tol, (k, err)
    net.close()


@pytest.mark.parametrize("dims,radius", [((24, 20), 1), ((6, 10, 8), 1), ((16, 16), 2)])
def test_patch_features_match_oracle(dims, radius):
    rng = np.random.default_rng(len(dims) * 10 + radius)
    Q = 6
    npix = int(np.prod(dims))
    y = (rng.standard_normal((Q, npix)) + 1j * rng.standard_normal((Q, npix))).astype(np.complex64)
    y[:, 5] = 0  # a zero pixel
    y[0, 7] = 0  # a zero coil-0 entry (no rotation)
    yd = torch.from_numpy(y).cuda()
    K = (2 * radius + 1) ** len(dims)
    X = torch.empty((npix, K * 2 * Q), dtype=torch.float32, device="cuda")
    assert B.pisco_warm_start_patch_features(yd.data_ptr(), Q, dims, radius, X.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream) == B.PISCO_OK
    torch.cuda.synchronize()
    ref = M.patch_features(y.astype(np.complex128), dims, radius)
    assert np.abs(X.cpu().numpy() - ref).max() <= 2e-6 * np.abs(ref).max()


def test_adam_step_matches_oracle_and_backward_is_deterministic():
    n_io, H, B = 16, 128, 1000
    rng = np.random.default_rng(3)
    p = he_init(n_io, H, n_io, seed=3)
    net = WarmStartNet(n_io // 2, H, params=p, max_batch=2048)
    x = torch.from_numpy(rng.standard_normal((B, n_io)).astype(np.float32)).cuda()
    t = torch.from_numpy(rng.standard_normal((B, n_io)).astype(np.float32)).cuda()
    net.backward(x, t)
    g1 = net.grads()
    net.backward(x, t)
    g2 = net.grads()
    np.testing.assert_array_equal(g1, g2)
    net.adam(1e-3)
    P = M.unpack(p, n_io, H, n_io)
    G = M.unpack(g1, n_io, H, n_io)
    m = {k: np.zeros(v.shape) for k, v in P.items()}
    v = {k: np.zeros(v.shape) for k, v in P.items()}
    exp = M.pack(M.adam_step(P, {k: G[k].astype(np.float64) for k in G}, m, v, 1, 1e-3))
    got = net.params()
    assert np.abs(got - exp).max() <= 2e-6
    net.close()


def test_training_reduces_loss_on_a_smooth_map():
    """Fit t = normalise(A x) for a fixed random A: the loss drops by an order of magnitude."""
    n_io, H, N = 16, 128, 32768
    rng = np.random.default_rng(5)
    A = rng.standard_normal((n_io, n_io)) / np.sqrt(n_io)
    x = rng.standard_normal((N, n_io))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    t = x @ A.T
    t /= np.linalg.norm(t, axis=1, keepdims=True)
    net = WarmStartNet(n_io // 2, H, seed=1, max_batch=4096, loss="mse")
    X = torch.from_numpy(x.astype(np.float32)).cuda()
    T = torch.from_numpy(t.astype(np.float32)).cuda()
    hist = net.fit(X, T, epochs=12, batch=1024, lr=2e-3, seed=0)
    print("loss per epoch:", [f"{h:.4f}" for h in hist])
    assert hist[-1] < 0.2 * hist[0]
    net.close()


def test_unequal_widths_have_no_skip_term():
    n_in, H, n_out, Bn = 12, 40, 7, 300
    rng = np.random.default_rng(11)
    p = he_init(n_in, H, n_out, seed=2) + 0.01
    st, h = B.pisco_mlp_create(n_in, H, n_out, p, 512, torch.cuda.current_stream().cuda_stream)
    assert st == B.PISCO_OK
    x = rng.standard_normal((Bn, n_in)).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty((Bn, n_out), dtype=torch.float32, device="cuda")
    assert B.pisco_mlp_forward(h, xd.data_ptr(), Bn, out.data_ptr()) == B.PISCO_OK
    torch.cuda.synchronize()
    ref, _ = M.forward(M.unpack(p, n_in, H, n_out), x)
    _close(out.cpu().numpy(), ref)
    B.pisco_mlp_destroy(h)
