"""Pins of the warm-start network's FP64 oracle (oracle/mlp_oracle.py) by mathematics alone:
central finite differences, closed forms of degenerate networks, one Adam step."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _rand_params(rng, n_in, H, n_out, scale=0.7):
    return {k: rng.standard_normal(s) * scale for k, s in M.shapes(n_in, H, n_out).items()}


@pytest.mark.parametrize("n_out", [3, 4])
def test_gradient_matches_central_differences(n_out):
    rng = np.random.default_rng(0)
    n_in, H, B = 4, 5, 7
    p = _rand_params(rng, n_in, H, n_out)
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal((B, n_out))
    L, g = M.backward(p, x, t, round16=False)
    assert abs(L - M.loss(p, x, t, round16=False)) < 1e-12
    h = 1e-6
    for k in M.LAYERS:
        flat = p[k].reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, x, t, round16=False)
            flat[idx] = old - h
            lm = M.loss(p, x, t, round16=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


@pytest.mark.parametrize("n_out", [6, 5])
def test_zero_weights_closed_form(n_out):
    """W1 = W2 = W3 = 0: the hidden units are the constants relu(b1), relu(b2), the output is
    b3 (+ x when the widths agree: the skip term); only W3 and b3 receive gradient:
    g_b3 = 2 mean(out - t), g_W3 = g_b3 relu(b2)^T."""
    rng = np.random.default_rng(1)
    n_in, H, B = 6, 8, 11
    p = {k: np.zeros(s) for k, s in M.shapes(n_in, H, n_out).items()}
    p["b1"] = rng.standard_normal(H)
    p["b2"] = rng.standard_normal(H)
    p["b3"] = rng.standard_normal(n_out)
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal((B, n_out))
    L, g = M.backward(p, x, t)
    out = p["b3"][None] + (x if n_out == n_in else 0.0)
    assert np.isclose(L, np.mean(np.sum((out - t) ** 2, axis=1)))
    gb3 = 2 * (out - t).mean(axis=0)
    np.testing.assert_allclose(g["b3"], gb3, atol=1e-12)
    np.testing.assert_allclose(g["W3"], np.outer(gb3, np.maximum(p["b2"], 0)), atol=1e-12)
    for k in ("W1", "b1", "W2", "b2"):
        assert np.all(g[k] == 0), k


def test_weights_are_evaluated_in_fp16():
    rng = np.random.default_rng(2)
    p = M.init_params(6, 8, 6, seed=3)
    x = rng.standard_normal((5, 6))
    out16, _ = M.forward(p, x)
    p16 = {k: (p[k].astype(np.float16).astype(np.float64) if k.startswith("W") else p[k]) for k in p}
    ref, _ = M.forward(p16, x, round16=False)
    np.testing.assert_array_equal(out16, ref)


def test_first_adam_step_is_a_signed_step():
    """From zero moments the bias-corrected first step is lr * g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    p = M.init_params(4, 5, 3, seed=5)
    g = {k: rng.standard_normal(v.shape) for k, v in p.items()}
    m = {k: np.zeros_like(v, dtype=np.float64) for k, v in p.items()}
    v = {k: np.zeros_like(v, dtype=np.float64) for k, v in p.items()}
    lr, eps = 1e-2, 1e-8
    new = M.adam_step(p, g, m, v, 1, lr, eps=eps)
    for k in M.LAYERS:
        exp = (p[k].astype(np.float64) - lr * g[k] / (np.abs(g[k]) + eps)).astype(np.float32)
        np.testing.assert_array_equal(new[k], exp)


def test_pack_unpack_and_features():
    p = M.init_params(8, 16, 8, seed=6)
    q = M.unpack(M.pack(p), 8, 16, 8)
    for k in M.LAYERS:
        np.testing.assert_array_equal(p[k], q[k])
    rng = np.random.default_rng(7)
    y = rng.standard_normal((9, 4)) + 1j * rng.standard_normal((9, 4))
    y[3] = 0
    x = M.features(y)
    np.testing.assert_allclose(np.linalg.norm(x, axis=1)[[0, 1, 2, 4]], 1.0)
    assert np.all(x[3] == 0)
    np.testing.assert_allclose(M.to_complex(x)[0] * np.linalg.norm(y[0]), y[0])


def test_zero_last_layer_starts_at_the_heuristic():
    """With W3 = 0 and b3 = 0 the network returns its input (the normalised low-res vector)."""
    p = M.init_params(8, 16, 8, seed=8, last_scale=0.0)
    x = np.random.default_rng(9).standard_normal((5, 8))
    out, _ = M.forward(p, x)
    np.testing.assert_array_equal(out, x)
