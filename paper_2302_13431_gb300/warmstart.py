"""Learned warm start of the per-pixel power iteration (an addition of this library: the paper
starts every pixel from an arbitrary vector, Sec. V-E).

A per-pixel MLP maps the patch of normalised low-resolution coil vectors around the pixel (the
apodised low-resolution images of Sec. V-D, which the estimate computes anyway; (2r+1)^D
neighbours, each divided by the centre's norm and rotated by the centre's coil-0 phase) to a
start vector for the power iteration: out = s(x) + W3 h2 + b3, a learned correction of the
heuristic start s(x) = y(x)/||y(x)|| (the patch's middle block).  The neighbourhood is what lets
the network see how the blur of rho c by the low-resolution kernel bends y away from c.
Training pairs come from the method itself: a teacher estimate with many power iterations gives
the converged null vector v(x) at every reduced-grid pixel; the loss is the phase-free direction
loss 1 - |<o, v>| / (||o|| ||v||).  Every forward, backward and update step runs in the library's
CUDA kernels through the C ABI (pisco_mlp_*; the layer products on the tensor cores); this module
only schedules them and moves tensors.

In the estimate, the proposal replaces the counter-based start; after `iters` iterations a
pixel whose residual ||G v - lambda |Lambda| v|| / |Lambda| exceeds `gate` is re-solved from
the plain start with the full iteration count (pisco_set_warm_start).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B
from .estimator import PiscoEstimator

LAYERS = ("W1", "b1", "W2", "b2", "W3", "b3")


def he_init(n_in, hidden, n_out, seed=0, last_scale=1.0):
    """Seeded initial parameters (the random numbers are inputs of the training): He-normal
    weights with std sqrt(2/fan_in) (the last layer scaled by last_scale), zero biases; FP32
    blob [W1|b1|W2|b2|W3|b3]."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (rows, cols) in enumerate(((hidden, n_in), (hidden, hidden), (n_out, hidden))):
        sc = last_scale if li == 2 else 1.0
        parts.append((rng.standard_normal((rows, cols)) * np.sqrt(2.0 / cols) * sc).astype(np.float32).reshape(-1))
        parts.append(np.zeros(rows, np.float32))
    return np.concatenate(parts)


class WarmStartNet:
    """Device-resident MLP (2r+1)^D 2Q -> hidden -> hidden -> 2Q (radius r, D = ndim)."""

    def __init__(self, Q, hidden=128, seed=0, params=None, max_batch=1 << 16, stream=None, radius=0, ndim=2,
                 loss="direction"):
        if not torch.cuda.is_available():
            raise RuntimeError("WarmStartNet needs a CUDA GPU (no CPU fallback)")
        self.Q, self.hidden, self.n_io = int(Q), int(hidden), 2 * int(Q)
        self.radius, self.ndim = int(radius), int(ndim)
        self.n_in = (2 * self.radius + 1) ** self.ndim * self.n_io
        self.max_batch = int(max_batch)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        # a zero last layer: the untrained network proposes the heuristic start y/||y|| itself
        p = (he_init(self.n_in, self.hidden, self.n_io, seed, last_scale=0.0) if params is None
             else np.asarray(params, np.float32))
        self.nparam = p.size
        st, h = B.pisco_mlp_create(self.n_in, self.hidden, self.n_io, p, self.max_batch, self.stream.cuda_stream)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_create")
        self._h = h
        self.set_loss(loss)

    def set_loss(self, loss):
        """"mse" (squared error to the target) or "direction" (phase-free direction loss)."""
        st = B.pisco_mlp_set_loss(self._h, {"mse": 0, "direction": 1}[loss])
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_set_loss")
        self.loss = loss

    # --------------------------------------------------------------------------------------
    def params(self) -> np.ndarray:
        st, p = B.pisco_mlp_read(self._h, 0, self.nparam)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_read")
        return p

    def grads(self) -> np.ndarray:
        st, g = B.pisco_mlp_read(self._h, 1, self.nparam)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_read")
        return g

    def set_params(self, params):
        st = B.pisco_mlp_write(self._h, params)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_write")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        x = x.contiguous()
        out = torch.empty((x.shape[0], self.n_io), dtype=torch.float32, device=x.device)
        for s in range(0, x.shape[0], self.max_batch):
            e = min(x.shape[0], s + self.max_batch)
            st = B.pisco_mlp_forward(self._h, x[s:e].data_ptr(), e - s, out[s:e].data_ptr())
            if st != B.PISCO_OK:
                raise B.PiscoError(st, "pisco_mlp_forward")
        return out

    def backward(self, x: torch.Tensor, t: torch.Tensor, want_loss=True):
        st, loss = B.pisco_mlp_backward(self._h, x.data_ptr(), t.data_ptr(), x.shape[0], want_loss)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_backward")
        return loss

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        st = B.pisco_mlp_adam(self._h, lr, beta1, beta2, eps)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_mlp_adam")

    def direction_error(self, X: torch.Tensor, T: torch.Tensor) -> float:
        """Median over samples of 1 - |<o, t>| / (||o|| ||t||) for the complex vectors o = net(x)
        and t: the phase-free distance of the proposal from the target direction (what the power
        iteration cares about)."""
        o = torch.view_as_complex(self.forward(X).reshape(X.shape[0], -1, 2).contiguous())
        t = torch.view_as_complex(T.reshape(T.shape[0], -1, 2).contiguous())
        c = (o.conj() * t).sum(dim=1).abs() / (o.abs().pow(2).sum(dim=1).sqrt() * t.abs().pow(2).sum(dim=1).sqrt()
                                                + 1e-30)
        return float((1.0 - c).median().item())

    def fit(self, X: torch.Tensor, T: torch.Tensor, epochs=10, batch=4096, lr=1e-3, seed=0, log_every=0,
            val=None):
        """Mini-batch Adam on (X, T); the sample order of each epoch is a seeded permutation.
        With val = (Xv, Tv), the parameters (including the initial ones) with the smallest
        validation direction_error are kept at the end.  Returns the mean loss of every epoch."""
        n = X.shape[0]
        gen = torch.Generator(device=X.device)
        gen.manual_seed(seed)
        hist = []
        best = None
        if val is not None:
            best = (self.direction_error(*val), self.params())
        self.val_history = [best[0]] if best else []
        for ep in range(epochs):
            perm = torch.randperm(n, generator=gen, device=X.device)
            tot, cnt = 0.0, 0
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                xb, tb = X.index_select(0, idx).contiguous(), T.index_select(0, idx).contiguous()
                want = log_every > 0 or s + 2 * batch > n
                loss = self.backward(xb, tb, want_loss=want)
                self.adam(lr)
                if loss is not None:
                    tot += loss
                    cnt += 1
            hist.append(tot / max(cnt, 1))
            if val is not None:
                e = self.direction_error(*val)
                self.val_history.append(e)
                if e < best[0]:
                    best = (e, self.params())
        if val is not None:
            self.set_params(best[1])
        return hist

    def attach(self, est: PiscoEstimator, iters: int, gate: float, fallback_iters: int):
        """Start `est`'s power iteration from this network's proposals (copied into the plan)."""
        st = B.pisco_set_warm_start(est._plan, self._h, iters, gate, fallback_iters)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_set_warm_start")

    def save(self, path):
        np.savez(path, params=self.params(), Q=self.Q, hidden=self.hidden, radius=self.radius, ndim=self.ndim)

    @classmethod
    def load(cls, path, **kw):
        z = np.load(path)
        r = int(z["radius"]) if "radius" in z.files else 0
        d = int(z["ndim"]) if "ndim" in z.files else 2
        return cls(int(z["Q"]), int(z["hidden"]), params=z["params"], radius=r, ndim=d, **kw)

    def close(self):
        if getattr(self, "_h", None):
            B.pisco_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def features(est: PiscoEstimator, radius=0) -> torch.Tensor:
    """Network inputs [npix_red, (2r+1)^D 2Q] from the low-resolution images of est's last
    estimate (the features the estimate itself computes for an attached network)."""
    Y = est.debug_buffer(B.PISCO_BUF_Y)
    npix = Y.numel() // est.Q
    K = (2 * radius + 1) ** len(est.reduced)
    X = torch.empty((npix, K * 2 * est.Q), dtype=torch.float32, device="cuda")
    st = B.pisco_warm_start_patch_features(Y.data_ptr(), est.Q, est.reduced, radius, X.data_ptr(),
                                           est.stream.cuda_stream)
    if st != B.PISCO_OK:
        raise B.PiscoError(st, "pisco_warm_start_patch_features")
    est.stream.synchronize()
    return X


def targets(est: PiscoEstimator) -> torch.Tensor:
    """Phase-aligned null vectors [npix_red, 2Q] (interleaved) of est's last estimate."""
    V = est.debug_buffer(B.PISCO_BUF_V).view(est.Q, -1)
    return torch.view_as_real(V.t().contiguous()).reshape(V.shape[1], 2 * est.Q).contiguous()


def _direction_gap(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """1 - |<a, b>| / (||a|| ||b||) per row of two interleaved [n, 2Q] arrays."""
    ac = torch.view_as_complex(a.reshape(a.shape[0], -1, 2).contiguous())
    bc = torch.view_as_complex(b.reshape(b.shape[0], -1, 2).contiguous())
    c = (ac.conj() * bc).sum(1).abs() / (ac.abs().pow(2).sum(1).sqrt() * bc.abs().pow(2).sum(1).sqrt() + 1e-30)
    return 1.0 - c


def teacher_pairs(teacher: PiscoEstimator, calibs, eig_max=0.05, radius=0, check: PiscoEstimator = None,
                  tol=1e-9):
    """Training pairs from the method itself: for every calibration block, the teacher's
    (features, converged null vector) at the reduced pixels whose eigenvalue lambda_min/|Lambda|
    is below eig_max (inside the object, where the null vector is the coil-map direction).
    check: the same estimator with fewer power iterations; a pixel whose two vectors differ by
    more than tol in direction has not converged (a near-degenerate null eigenvalue: no unique
    target) and is left out."""
    xs, ts = [], []
    for c in calibs:
        maps, eig = teacher(c)
        ok = eig.reshape(-1) < eig_max
        if check is not None:
            check(c)
            ok &= _direction_gap(targets(check), targets(teacher)) < tol
        keep = ok.nonzero().reshape(-1)
        xs.append(features(teacher, radius).index_select(0, keep))
        ts.append(targets(teacher).index_select(0, keep))
    return torch.cat(xs), torch.cat(ts)


def generated_pairs(teacher: PiscoEstimator, seeds, eig_max=0.05, radius=0, check=None, **gen):
    """teacher_pairs over volumes drawn by phantoms_torch.make_calib (one volume on the device at
    a time); gen: grid, Q, calib_shape and the generator's options."""
    from .phantoms_torch import make_calib
    xs, ts = [], []
    for s in seeds:
        calib, _ = make_calib(gen["grid"], gen["Q"], gen["calib_shape"], seed=int(s),
                              **{k: v for k, v in gen.items() if k not in ("grid", "Q", "calib_shape")})
        x, t = teacher_pairs(teacher, [calib], eig_max=eig_max, radius=radius, check=check)
        xs.append(x)
        ts.append(t)
        del calib
    return torch.cat(xs), torch.cat(ts)


def train_warm_start(grid, Q, calib_shape, tau, reduction, train_seeds, val_seeds, kernel_shape="ellipsoid",
                     hidden=128, epochs=6, batch=8192, lr=5e-4, teacher_iters=400, seed=0, log=None, radius=1):
    """Train a warm-start network (patch radius `radius`) on volumes the estimator itself labels
    (teacher: the same estimator with teacher_iters power iterations) with the direction loss,
    and select it on the validation volumes.  Returns (net, info)."""
    teacher = PiscoEstimator(grid, calib_shape, Q, tau, kernel_shape=kernel_shape, reduction=reduction,
                             iters=teacher_iters)
    check = PiscoEstimator(grid, calib_shape, Q, tau, kernel_shape=kernel_shape, reduction=reduction,
                           iters=teacher_iters // 2)
    gen = dict(grid=grid, Q=Q, calib_shape=calib_shape)
    X, T = generated_pairs(teacher, train_seeds, radius=radius, check=check, **gen)
    Xv, Tv = generated_pairs(teacher, val_seeds, radius=radius, check=check, **gen)
    teacher.close()
    check.close()
    net = WarmStartNet(Q, hidden, seed=seed, max_batch=batch, radius=radius, ndim=len(grid))
    hist = net.fit(X, T, epochs=epochs, batch=batch, lr=lr, seed=seed, val=(Xv, Tv))
    info = dict(train_pairs=int(X.shape[0]), val_pairs=int(Xv.shape[0]), loss=hist,
                val_direction_error=net.val_history, train_volumes=len(train_seeds),
                val_volumes=len(val_seeds))
    if log:
        log(info)
    return net, info
