"""FP64 CPU oracle of the learned warm start's network (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may use this module;
the product path never does.

The warm start proposes each pixel's power-iteration start vector (Sec. V-E) from the pixel's
normalised low-resolution coil vector y(x)/||y(x)|| (Sec. V-D) with a small per-pixel MLP:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  out = x + W3 h2 + b3

x and out are 2Q reals (real and imaginary parts interleaved per coil), the hidden layers have
H units.  The skip term x (present whenever the input and output widths agree) makes the
network a learned correction of the heuristic start y(x)/||y(x)||.  Weights are stored in FP16 (biases FP32); the oracle evaluates the FP16-rounded
weights in FP64.  Loss: mean over the batch of the squared error to the target vector,
L = (1/B) sum_b ||out_b - t_b||^2.  Optimiser: Adam with bias correction (Kingma & Ba, 2015)
on FP32 master weights.

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


def forward(p, x, round16=True):
    """x: [B, n_in].  Returns out [B, n_out] and the cache of pre-activations/activations."""
    e = effective(p, round16)
    x = np.asarray(x, np.float64)
    z1 = x @ e["W1"].T + e["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ e["W2"].T + e["b2"]
    h2 = np.maximum(z2, 0.0)
    out = h2 @ e["W3"].T + e["b3"]
    if x.shape[1] == out.shape[1]:
        out = out + x
    return out, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2)


def loss(p, x, t, round16=True):
    out, _ = forward(p, x, round16)
    return float(np.sum((out - t) ** 2) / x.shape[0])


def backward(p, x, t, round16=True):
    """Loss and its gradient with respect to every parameter (chain rule, layer by layer).
    With FP16 weights the gradient is taken with respect to the evaluated (rounded) weights
    and applied to the FP32 masters."""
    e = effective(p, round16)
    out, c = forward(p, x, round16)
    B = x.shape[0]
    d_out = 2.0 * (out - np.asarray(t, np.float64)) / B
    g = {}
    g["W3"] = d_out.T @ c["h2"]
    g["b3"] = d_out.sum(axis=0)
    d_h2 = d_out @ e["W3"]
    d_z2 = d_h2 * (c["z2"] > 0)
    g["W2"] = d_z2.T @ c["h1"]
    g["b2"] = d_z2.sum(axis=0)
    d_h1 = d_z2 @ e["W2"]
    d_z1 = d_h1 * (c["z1"] > 0)
    g["W1"] = d_z1.T @ c["x"]
    g["b1"] = d_z1.sum(axis=0)
    return float(np.sum((out - t) ** 2) / B), g


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


def features(y):
    """Network input from low-resolution coil vectors y [npix, Q] (complex): y/||y||, real and
    imaginary parts interleaved per coil; zero vectors stay zero."""
    y = np.asarray(y, np.complex128)
    n = np.linalg.norm(y, axis=1, keepdims=True)
    u = np.where(n > 0, y / np.where(n > 0, n, 1.0), 0.0)
    x = np.empty((y.shape[0], 2 * y.shape[1]))
    x[:, 0::2] = u.real
    x[:, 1::2] = u.imag
    return x


def to_complex(out):
    """[npix, 2Q] interleaved reals -> [npix, Q] complex."""
    return out[:, 0::2] + 1j * out[:, 1::2]
