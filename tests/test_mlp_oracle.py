"""Pins of the warm-start network's FP64 oracle (oracle/mlp_oracle.py) by mathematics alone:
central finite differences (both losses), closed forms of degenerate networks, invariances of
the direction loss and of the patch features, FP16 rounding as a no-op on FP16-exact data, one
Adam step."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _rand_params(rng, n_in, H, n_out, scale=0.7):
    return {k: rng.standard_normal(s) * scale for k, s in M.shapes(n_in, H, n_out).items()}


@pytest.mark.parametrize("n_in,n_out,kind", [(4, 3, 0), (4, 4, 0), (12, 4, 0), (4, 4, 1), (12, 4, 1), (6, 4, 1)])
def test_gradient_matches_central_differences(n_in, n_out, kind):
    """Both losses; skip term absent (4 -> 3, 6 -> 4), the whole input (4 -> 4) or the middle
    block (12 -> 4)."""
    rng = np.random.default_rng(n_in + n_out + kind)
    H, B = 5, 7
    p = _rand_params(rng, n_in, H, n_out)
    x = rng.standard_normal((B, n_in))
    t = rng.standard_normal((B, n_out))
    L, g = M.backward(p, x, t, round16=False, kind=kind)
    assert abs(L - M.loss(p, x, t, round16=False, kind=kind)) < 1e-12
    h = 1e-6
    for k in M.LAYERS:
        flat = p[k].reshape(-1)
        for idx in range(flat.size):
            old = flat[idx]
            flat[idx] = old + h
            lp = M.loss(p, x, t, round16=False, kind=kind)
            flat[idx] = old - h
            lm = M.loss(p, x, t, round16=False, kind=kind)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].reshape(-1)[idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (k, idx)


def test_direction_loss_is_phase_and_scale_free():
    rng = np.random.default_rng(12)
    o = rng.standard_normal((6, 8))
    t = rng.standard_normal((6, 8))
    l0, _ = M.sample_losses(o, t, 1)
    oc = M.to_complex(o) * (2.5 * np.exp(1j * rng.uniform(0, 6.3, (6, 1))))
    o2 = np.empty_like(o)
    o2[:, 0::2], o2[:, 1::2] = oc.real, oc.imag
    l1, _ = M.sample_losses(o2, t, 1)
    np.testing.assert_allclose(l0, l1, atol=1e-13)
    tc = M.to_complex(t) * (0.3 - 1.1j)  # o parallel to t: loss 0, gradient 0
    tt = np.empty_like(t)
    tt[:, 0::2], tt[:, 1::2] = tc.real, tc.imag
    l2, d2 = M.sample_losses(t, tt, 1)
    assert np.abs(l2).max() < 1e-14 and np.abs(d2).max() < 1e-12
    assert np.all((l0 >= 0) & (l0 <= 1))


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
    L, g = M.backward(p, x, t, round16=False)
    out = p["b3"][None] + (x if n_out == n_in else 0.0)
    assert np.isclose(L, np.mean(np.sum((out - t) ** 2, axis=1)))
    gb3 = 2 * (out - t).mean(axis=0)
    np.testing.assert_allclose(g["b3"], gb3, atol=1e-12)
    np.testing.assert_allclose(g["W3"], np.outer(gb3, np.maximum(p["b2"], 0)), atol=1e-12)
    for k in ("W1", "b1", "W2", "b2"):
        assert np.all(g[k] == 0), k


def test_fp16_rounding_is_exact_on_fp16_data_and_rounds_otherwise():
    """Weights, inputs and biases on a grid of 1/8 with small integer hidden sums: every product
    operand is an FP16 number, so the rounded evaluation equals the exact one; generic data
    differs by the FP16 rounding (about 2^-11 relative)."""
    rng = np.random.default_rng(2)
    p = {k: rng.integers(-4, 5, s) / 8.0 for k, s in M.shapes(6, 8, 6).items()}
    x = rng.integers(-4, 5, (5, 6)) / 8.0
    out16, _ = M.forward(p, x)
    ref, _ = M.forward(p, x, round16=False)
    np.testing.assert_array_equal(out16, ref)
    p = M.init_params(6, 8, 6, seed=3)
    x = rng.standard_normal((5, 6))
    a, _ = M.forward(p, x)
    b, _ = M.forward(p, x, round16=False)
    err = np.abs(a - b).max() / np.abs(b).max()
    assert 1e-6 < err < 1e-2


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
    rot = np.conj(y[0, 0]) / abs(y[0, 0])
    np.testing.assert_allclose(M.to_complex(x)[0] * np.linalg.norm(y[0]), y[0] * rot)
    np.testing.assert_allclose(M.to_complex(x)[0, 0].imag, 0.0, atol=1e-15)  # coil 0 real positive


@pytest.mark.parametrize("dims,r", [((5, 7), 1), ((4, 3, 5), 1), ((6, 6), 2)])
def test_patch_features_centre_block_shift_and_constant_field(dims, r):
    rng = np.random.default_rng(len(dims) + r)
    Q = 3
    npix = int(np.prod(dims))
    y = rng.standard_normal((Q, npix)) + 1j * rng.standard_normal((Q, npix))
    K = (2 * r + 1) ** len(dims)
    x = M.patch_features(y, dims, r)
    assert x.shape == (npix, K * 2 * Q)
    # the centre block is the radius-0 feature; the skip offset points at it
    np.testing.assert_allclose(x[:, (K // 2) * 2 * Q:(K // 2 + 1) * 2 * Q], M.features(y.T))
    assert M.skip_offset(K * 2 * Q, 2 * Q) == (K // 2) * 2 * Q
    # periodic shift: rolling the images rolls the features
    sh = tuple(1 for _ in dims)
    ys = np.roll(y.reshape((Q,) + dims), sh, axis=tuple(range(1, len(dims) + 1))).reshape(Q, -1)
    xs = M.patch_features(ys, dims, r)
    xr = np.roll(x.reshape(dims + (-1,)), sh, axis=tuple(range(len(dims)))).reshape(npix, -1)
    np.testing.assert_allclose(xs, xr, atol=1e-14)
    # a constant field: every neighbour differs from the centre by nothing
    yc = np.repeat(y[:, :1], npix, axis=1)
    xc = M.patch_features(yc, dims, r).reshape(npix, K, 2 * Q)
    assert np.abs(np.delete(xc, K // 2, axis=1)).max() < 1e-15
    # a neighbour block plus the centre block is that neighbour's vector in the centre's frame
    xb = x.reshape(npix, K, 2 * Q)
    u = M.to_complex(xb[:, 0] + xb[:, K // 2])
    first = tuple(-r for _ in dims)
    nb = np.roll(y.reshape((Q,) + dims), tuple(-v for v in first), axis=tuple(range(1, len(dims) + 1))).reshape(Q, -1).T
    rot = np.conj(y[0]) / np.abs(y[0]) / np.linalg.norm(y, axis=0)
    np.testing.assert_allclose(u, nb * rot[:, None], atol=1e-13)


def test_zero_last_layer_starts_at_the_heuristic():
    """With W3 = 0 and b3 = 0 the network returns its input (the normalised low-res vector)."""
    p = M.init_params(8, 16, 8, seed=8, last_scale=0.0)
    x = np.random.default_rng(9).standard_normal((5, 8))
    out, _ = M.forward(p, x)
    np.testing.assert_array_equal(out, x)
