"""FP64 CPU oracle of the learned warm start's network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use this module;
the product path never does.

The warm start proposes each pixel's power-iteration start vector (Sec. V-E) from the patch of
normalised low-resolution coil vectors around the pixel (Sec. V-D) with a small per-pixel MLP:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  out = s(x) + W3 h2 + b3

x is the patch (patch_features: (2r+1)^D neighbours, each 2Q reals, real and imaginary parts
interleaved per coil), out 2Q reals, the hidden layers have H units.  The skip term s(x), the
middle block of x when n_in is an odd multiple of n_out (the centre pixel's own normalised
vector), makes the network a learned correction of the heuristic start y(x)/||y(x)||.

Precision: the products run with FP16 operands and FP32 accumulation; with round16 the oracle
rounds every product operand to FP16 (weights, the input x, the hidden activations, the
per-sample gradients) and evaluates the rest in FP64 (biases, ReLU, skip term, losses).
Losses (mean over the batch): the squared error ||out - t||^2, or the direction loss
1 - |<o, t>| / (||o|| ||t||) of the complex vectors (<o, t> = sum_q conj(o_q) t_q).  Gradients:
per-sample loss gradients d_b (unscaled), weight gradients (1/B) sum_b d_b^T a_b over the
rounded operands.  Optimiser: Adam with bias correction (Kingma & Ba, 2015) on FP32 master
weights.

The paper has no network: this part is an addition of this library, so every step here is
pinned by mathematics alone (finite differences, closed forms), not by a printed value.
"""
from __future__ import annotations

import numpy as np

LAYERS = ("W1", "b1", "W2", "b2", "W3", "b3")


def shapes(n_in, n_hidden, n_out):
    return {"W1": (n_hidden, n_in), "b1": (n_hidden,), "W2": (n_hidden, n_hidden), "b2": (n_hidden,),
            "W3": (n_out, n_hidden), "b3": (n_out,)}


def init_params(n_in, n_hidden, n_out, seed=0, last_scale=1.0):
    """He-normal weights (std sqrt(2/fan_in); W3 scaled by last_scale), zero biases, FP32."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in shapes(n_in, n_hidden, n_out).items():
        if name.startswith("W"):
            sc = last_scale if name == "W3" else 1.0
            p[name] = (rng.standard_normal(shp) * np.sqrt(2.0 / shp[1]) * sc).astype(np.float32)
        else:
            p[name] = np.zeros(shp, np.float32)
    return p


def pack(p):
    """Flat FP32 blob in LAYERS order (row-major weights)."""
    return np.concatenate([np.asarray(p[k], np.float32).reshape(-1) for k in LAYERS])


def unpack(blob, n_in, n_hidden, n_out):
    out, o = {}, 0
    for k in LAYERS:
        shp = shapes(n_in, n_hidden, n_out)[k]
        n = int(np.prod(shp))
        out[k] = np.asarray(blob[o:o + n], np.float32).reshape(shp)
        o += n
    return out


def effective(p, round16=True):
    """The weights the network evaluates: FP16-rounded matrices, FP32 biases, as FP64
    (round16=False keeps the matrices unrounded, for finite-difference checks)."""
    return {k: (np.asarray(p[k]).astype(np.float16).astype(np.float64) if (k.startswith("W") and round16)
                else np.asarray(p[k], np.float64)) for k in LAYERS}


def skip_offset(n_in, n_out):
    """Column offset of the skip term in x (the middle block), or None."""
    if n_in % n_out or (n_in // n_out) % 2 == 0:
        return None
    return (n_in // n_out // 2) * n_out


def _r16(a, on):
    a = np.asarray(a, np.float64)
    return a.astype(np.float32).astype(np.float16).astype(np.float64) if on else a


def forward(p, x, round16=True):
    """x: [B, n_in].  Returns out [B, n_out] and the cache of pre-activations/activations."""
    e = effective(p, round16)
    x = np.asarray(x, np.float64)
    z1 = _r16(x, round16) @ e["W1"].T + e["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = _r16(h1, round16) @ e["W2"].T + e["b2"]
    h2 = np.maximum(z2, 0.0)
    out = _r16(h2, round16) @ e["W3"].T + e["b3"]
    so = skip_offset(x.shape[1], out.shape[1])
    if so is not None:
        out = out + x[:, so:so + out.shape[1]]
    return out, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2)


def sample_losses(out, t, kind=0):
    """Per-sample losses and their gradients with respect to out (unscaled)."""
    out = np.asarray(out, np.float64)
    t = np.asarray(t, np.float64)
    if kind == 0:
        return np.sum((out - t) ** 2, axis=1), 2.0 * (out - t)
    o, tc = to_complex(out), to_complex(t)
    s = np.sum(np.conj(o) * tc, axis=1)
    a = np.abs(s)
    no, nt = np.linalg.norm(o, axis=1), np.linalg.norm(tc, axis=1)
    ok = (no > 0) & (nt > 0)
    den = np.where(ok, no * nt, 1.0)
    loss = np.where(ok, 1.0 - a / den, 0.0)
    ph = np.where(a > 0, np.conj(s) / np.where(a > 0, a, 1.0), 1.0)  # e^{-i arg s}
    # the gradient of |s| with respect to o (as the complex number d/dRe + i d/dIm) is
    # t e^{-i arg s}; that of ||o|| is o / ||o||
    gc = -(tc * ph[:, None] / np.where(ok, no, 1.0)[:, None]
           - (a / np.where(ok, no ** 3, 1.0))[:, None] * o) / np.where(ok, nt, 1.0)[:, None]
    gc = np.where(ok[:, None], gc, 0.0)
    d = np.empty_like(out)
    d[:, 0::2] = gc.real
    d[:, 1::2] = gc.imag
    return loss, d


def loss(p, x, t, round16=True, kind=0):
    out, _ = forward(p, x, round16)
    return float(np.mean(sample_losses(out, t, kind)[0]))


def backward(p, x, t, round16=True, kind=0):
    """Loss and its gradient with respect to every parameter (chain rule, layer by layer).
    With round16 the products take FP16-rounded operands as the kernels do (the gradient is
    then that of the kernels' arithmetic: taken with respect to the evaluated weights and
    applied to the FP32 masters)."""
    e = effective(p, round16)
    out, c = forward(p, x, round16)
    B = x.shape[0]
    ls, d_out = sample_losses(out, t, kind)
    r = lambda a: _r16(a, round16)
    g = {}
    g["W3"] = r(d_out).T @ r(c["h2"]) / B
    g["b3"] = r(d_out).sum(axis=0) / B
    d_h2 = r(d_out) @ e["W3"]
    d_z2 = d_h2 * (c["z2"] > 0)
    g["W2"] = r(d_z2).T @ r(c["h1"]) / B
    g["b2"] = r(d_z2).sum(axis=0) / B
    d_h1 = r(d_z2) @ e["W2"]
    d_z1 = d_h1 * (c["z1"] > 0)
    g["W1"] = r(d_z1).T @ r(c["x"]) / B
    g["b1"] = r(d_z1).sum(axis=0) / B
    return float(np.mean(ls)), g


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update of the FP32 master weights (step counts from 1).  m, v: moment dicts
    (updated in place).  Returns the new parameters."""
    new = {}
    for k in LAYERS:
        m[k] = beta1 * m[k] + (1 - beta1) * g[k]
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] ** 2
        mh = m[k] / (1 - beta1 ** step)
        vh = v[k] / (1 - beta2 ** step)
        new[k] = (p[k].astype(np.float64) - lr * mh / (np.sqrt(vh) + eps)).astype(np.float32)
    return new


def patch_features(y, dims, radius):
    """Network input from low-resolution coil images y [Q, npix] (complex) on the periodic grid
    dims (2 or 3 axes, x fastest): with u(k) = y(k) conj(y_0(j)) / (|y_0(j)| ||y(j)||), the centre
    block u(j) and, for every other neighbour o of the (2r+1)^D patch around pixel j (slowest
    axis first), u(j + o) - u(j); real and imaginary parts interleaved, [npix, (2r+1)^D * 2Q].
    A zero y_0(j) gives no rotation, a zero y(j) zeros."""
    y = np.asarray(y, np.complex128)
    Q = y.shape[0]
    img = y.reshape((Q,) + tuple(dims))
    n = np.linalg.norm(img, axis=0)
    a0 = np.abs(img[0])
    rot = np.where(a0 > 0, np.conj(img[0]) / np.where(a0 > 0, a0, 1.0), 1.0)
    scale = np.where(n > 0, rot / np.where(n > 0, n, 1.0), 0.0)
    D = len(dims)
    offs = [()]
    for _ in range(D):
        offs = [o + (d,) for o in offs for d in range(-radius, radius + 1)]
    blocks = []
    centre = (img * scale[None]).reshape(Q, -1).T
    for o in offs:
        nb = np.roll(img, tuple(-v for v in o), axis=tuple(range(1, D + 1)))  # nb[j] = img[j + o]
        u = (nb * scale[None]).reshape(Q, -1).T
        blocks.append(u if not any(o) else u - centre)
    z = np.stack(blocks, axis=1)  # [npix, K, Q]
    x = np.empty(z.shape[:2] + (2 * Q,))
    x[..., 0::2] = z.real
    x[..., 1::2] = z.imag
    return x.reshape(z.shape[0], -1)


def features(y):
    """Radius-0 features of low-resolution coil vectors y [npix, Q] (complex):
    y conj(y_0) / (|y_0| ||y||), real and imaginary parts interleaved per coil."""
    y = np.asarray(y, np.complex128)
    return patch_features(y.T, (1, y.shape[0]), 0)


def to_complex(out):
    """[npix, 2Q] interleaved reals -> [npix, Q] complex."""
    return out[:, 0::2] + 1j * out[:, 1::2]
