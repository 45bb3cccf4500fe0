"""The warm-start network's CUDA kernels (through the C ABI) against the FP64 oracle MLP:
forward pass, loss, every gradient, one Adam step; determinism of the batch reductions.
Tolerances: FP32 accumulation over <= 128 terms (forward) and over the batch (gradients)
against FP64 with the same FP16-rounded weights."""
import numpy as np
import pytest

from oracle import mlp_oracle as M

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.warmstart import WarmStartNet, he_init  # noqa: E402


@pytest.mark.parametrize("n_io,H,B", [(16, 128, 700), (64, 128, 4096), (10, 37, 129)])
def test_forward_loss_and_gradients_match_oracle(n_io, H, B):
    rng = np.random.default_rng(n_io + H + B)
    p = he_init(n_io, H, n_io, seed=n_io)
    p = p + (rng.standard_normal(p.size) * 0.05).astype(np.float32)
    net = WarmStartNet(n_io // 2, H, params=p, max_batch=4096)
    x = rng.standard_normal((B, n_io)).astype(np.float32)
    t = rng.standard_normal((B, n_io)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    out = net.forward(xd).cpu().numpy()
    P = M.unpack(p, n_io, H, n_io)
    ref, _ = M.forward(P, x)
    assert np.abs(out - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    loss = net.backward(xd, td)
    L, g = M.backward(P, x, t)
    assert abs(loss - L) <= 1e-5 * L
    gg = M.unpack(net.grads(), n_io, H, n_io)
    tol = 1e-4 * max(1.0, np.sqrt(B / 256))  # FP32 sums over the batch, fixed order
    for k in M.LAYERS:
        err = np.abs(gg[k] - g[k]).max() / max(np.abs(g[k]).max(), 1e-12)
        assert err <= tol, (k, err)
    net.close()


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
    net = WarmStartNet(n_io // 2, H, seed=1, max_batch=4096)
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
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-5 * max(1.0, np.abs(ref).max())
    B.pisco_mlp_destroy(h)
