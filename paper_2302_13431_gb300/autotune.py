"""Autotuner of the batched estimator's launch configuration.

For a batch of problem shapes it times every candidate configuration on the device, as a
captured batch (one CUDA-graph replay per step, the way the batch runs in production), and keeps
the fastest.  The knobs are ones whose best value depends on the shapes and on how many estimates
share the GPU:

* precision route: CUDA-core FP32 products, or split-TF32 tensor-core products for the G(x)
  assembly only, also for the eigensolver's A X products, or for every block product (all meet
  the FP32 parity gates; the one-pass TF32 routes do not and are never candidates);
* `tc_splits`: K splits of the tensor-core block products (more splits shorten one product,
  fewer cost less SM time and reduction traffic);
* `gemm_splits`: split-K cap of the CUDA-core block products (same trade-off);
* `gemm_tile`: 32x32 or 64x64 output tiles for those products (lower latency vs less SM time);
* `gram_df`: the Gram's FFT route in FP64 or in double-float arithmetic (pairs of FP32);
* `tc_interp`: the last interpolation pass as a batched split-TF32 tensor-core GEMM or as the
  fused CUDA-core interpolate-and-normalise kernel (tried on the best of the others only);
* `batch_group`: how many items of identical parameters one batched pass estimates (0: all of
  them, up to 64; 1: one launch chain per item; tried on the best of the others only).

A candidate counts only if it passes a correctness gate on the tuning batch: every item returns
PISCO_OK, with the same signal dimension as the first candidate (plain FP32) and eigenvalue maps
within 1e-4 of it; candidates that fail are listed with ms = None and never chosen.

Results are cached in a JSON file keyed by the device name, the shapes and the batch size.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import torch

from .estimator import PiscoBatch
from .phantoms import make_case

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")

KNOB_KEYS = ("precision", "tc_splits", "gemm_splits", "gemm_tile", "gram_df", "tc_interp", "batch_group")
# knobs toggled one at a time on the best candidate after the main sweep
REFINE = (("tc_interp", True), ("batch_group", 1), ("batch_group", 16), ("batch_group", 32))


def candidates():
    base = dict(tc_interp=False, batch_group=0)
    out = [dict(base, precision="fp32", tc_splits=0, gemm_splits=0, gemm_tile=0, gram_df=False),
           dict(base, precision="fp32", tc_splits=0, gemm_splits=2, gemm_tile=64, gram_df=False),
           dict(base, precision="tc_g", tc_splits=0, gemm_splits=2, gemm_tile=64, gram_df=False)]
    for df in (False, True):
        for ts in (1, 4):
            for gs, gt in ((0, 0), (2, 64)):
                out.append(dict(base, precision="tc_g_eig", tc_splits=ts, gemm_splits=gs, gemm_tile=gt, gram_df=df))
            out.append(dict(base, precision="tc_all", tc_splits=ts, gemm_splits=0, gemm_tile=0, gram_df=df))
    return out


def _shape_key(specs, batch_note=""):
    shapes = [(tuple(s["grid"]), tuple(s["calib_shape"]), s["num_coils"], s["tau"] if isinstance(s["tau"], int)
               else tuple(s["tau"]), s.get("kernel_shape", "ellipsoid"), s.get("reduction", 1), s.get("iters", 30))
              for s in specs]
    h = hashlib.sha1(repr(shapes).encode()).hexdigest()[:16]
    dev = torch.cuda.get_device_name(0) if torch.cuda.is_available() else "cpu"
    return f"{dev}|{len(specs)} items|{h}{batch_note}"


def _time_batch(specs, calibs, steps, warmup, ref=None):
    """(ms per step, outputs) of one candidate, or (None, reason) when it fails the gate against
    `ref` (the outputs of the reference candidate: per-item signal dimensions and eigenvalue maps)."""
    from . import _binding as B
    batch = PiscoBatch(specs)
    maps, eigs = batch.alloc_outputs()
    try:
        try:
            for _ in range(warmup):
                batch.estimate_into(calibs, maps, eigs)
        except B.PiscoError as e:
            return None, f"batch call failed: {e}"
        torch.cuda.synchronize()
        st = list(batch.last_item_status)
        if any(x != B.PISCO_OK for x in st):
            return None, f"item statuses {st}"
        ks = [batch.item_stats(i)["signal_dim"] for i in range(len(specs))]
        out = (ks, [e.clone() for e in eigs])
        if ref is not None:
            if ks != ref[0]:
                return None, f"signal dims {ks} != {ref[0]}"
            d = max(float((a - b).abs().max()) for a, b in zip(eigs, ref[1]))
            if not d <= 1e-4:
                return None, f"eigenvalue maps differ by {d:.2e}"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            batch.estimate_into(calibs, maps, eigs)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out
    finally:
        batch.close()


def tune(specs, calibs=None, steps=3, warmup=2, cache=DEFAULT_CACHE, cands=None, refresh=False, verbose=False,
         refine=None):
    """Best configuration (dict of KNOB_KEYS) for the batch `specs` (PiscoBatch spec dicts).

    calibs: device calibration tensors (synthetic ones are generated when None).  refine: the
    (knob, value) toggles tried on the best candidate of the sweep (default REFINE).  Returns
    (config, table) where table lists every candidate with its milliseconds per batch step."""
    refine = REFINE if refine is None else tuple(refine)
    key = _shape_key(specs) + ("" if refine == REFINE else "|refine=" + json.dumps(refine))
    db = {}
    if cache and os.path.exists(cache):
        try:
            with open(cache) as f:
                db = json.load(f)
        except Exception:
            db = {}
    if not refresh and key in db:
        return db[key]["config"], db[key]["table"]
    if calibs is None:
        calibs = [torch.from_numpy(make_case(s["grid"], s["num_coils"], s["calib_shape"], seed=7000 + i).calib).cuda()
                  for i, s in enumerate(specs)]
    table = []
    t0 = time.time()
    ref = None
    for c in (cands or candidates()):
        sp = [dict(s, **c) for s in specs]
        ms, out = _time_batch(sp, calibs, steps, warmup, ref)
        table.append(dict(c, ms=ms) if ms is not None else dict(c, ms=None, rejected=out))
        if ms is not None and ref is None:
            ref = out
        if verbose:
            print(f"  autotune {c}: {ms if ms is None else round(ms, 3)} ms/step", flush=True)
    ok = [r for r in table if r["ms"] is not None]
    if not ok:
        raise RuntimeError("autotune: no candidate passed the correctness gate: " + repr(table))
    best = min(ok, key=lambda r: r["ms"])
    if cands is None:
        for knob, val in refine:
            c = {k: best[k] for k in KNOB_KEYS}
            if c[knob] == val:
                continue
            c[knob] = val
            ms, out = _time_batch([dict(s, **c) for s in specs], calibs, steps, warmup, ref)
            table.append(dict(c, ms=ms) if ms is not None else dict(c, ms=None, rejected=out))
            if verbose:
                print(f"  autotune {c}: {ms} ms/step", flush=True)
            if ms is not None and ms < best["ms"]:
                best = table[-1]
    config = {k: best[k] for k in KNOB_KEYS}
    if cache:
        db[key] = dict(config=config, table=table, seconds=time.time() - t0)
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        with open(cache, "w") as f:
            json.dump(db, f, indent=1)
    return config, table


def apply(specs, config):
    """The batch specs with the tuned knobs set."""
    return [dict(s, **config) for s in specs]
