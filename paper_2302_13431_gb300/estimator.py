"""torch-facing wrapper of the PISCO C ABI.

torch provides device memory and the CUDA stream; every step of the estimator runs in the
CUDA library (see include/pisco.h).  There is no CPU fallback: constructing an estimator
without the library or without a GPU raises.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _binding as B


class _DevView:
    """Exposes a raw device pointer through __cuda_array_interface__ for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 2}


PRECISIONS = {
    # name: (flags, meaning)
    "fp32": (0, "CUDA-core FP32 products everywhere (the plain path)"),
    "tc_g": (B.PISCO_FLAG_TC_GFIELD, "G(x) assembly on tensor cores, 3-pass split TF32"),
    "tc_g_eig": (B.PISCO_FLAG_TC_GFIELD | B.PISCO_FLAG_TC_EIG,
                 "G(x) assembly and eigensolver block products on tensor cores, 3-pass split TF32"),
    "tc_all": (B.PISCO_FLAG_TC_GFIELD | B.PISCO_FLAG_TC_EIG | B.PISCO_FLAG_TC_THIN,
               "G(x) assembly and every eigensolver block product on tensor cores, 3-pass split TF32"),
    "tc_g_1pass": (B.PISCO_FLAG_TC_GFIELD | B.PISCO_FLAG_TC_1PASS, "G(x) assembly, single TF32 pass"),
    "tc_g_eig_1pass": (B.PISCO_FLAG_TC_GFIELD | B.PISCO_FLAG_TC_EIG | B.PISCO_FLAG_TC_1PASS,
                       "G(x) and eigensolver products, single TF32 pass"),
}


def precision_flags(precision: str) -> int:
    if precision not in PRECISIONS:
        raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
    return PRECISIONS[precision][0]


class PiscoEstimator:
    """One plan of the estimator for a fixed problem shape.

    grid, calib_shape: (z,)y,x sizes of the image grid and the centred calibration box.
    tau: radius (int or per-axis tuple); kernel_shape: "ellipsoid" (Sec. V-B) or "rect".
    reduction: grid-reduction factor f (Sec. V-D); iters: power iterations (Sec. V-E).
    masked_gram: the exact Gram of the masked calibration matrix instead of Sec. V-A's FFT route.
    block_pi: two-vector block power iteration with Rayleigh-Ritz (small-gap pixels).
    gram_df: the Gram's FFT route in double-float instead of FP64 arithmetic.
    tc_interp: the last interpolation pass as one batched split-TF32 tensor-core GEMM.
    g_dense: with a tensor-core G(x) route in 2D, the dense lag product instead of the separable
    DFT passes.
    """

    def __init__(self, grid, calib_shape, num_coils, tau, kernel_shape="ellipsoid", thr=0.05,
                 reduction=1, iters=30, seed=0, host_io=False, eig_block=0, eig_iters=0,
                 stream=None, precision="fp32", tc_splits=0, gemm_splits=0, masked_gram=False,
                 block_pi=False, gemm_tile=0, gram_df=False, tc_interp=False,
                 g_dense=False):
        if not torch.cuda.is_available():
            raise RuntimeError("PiscoEstimator needs a CUDA GPU (no CPU fallback)")
        self.grid = tuple(int(g) for g in grid)
        self.calib_shape = tuple(int(c) for c in calib_shape)
        self.Q = int(num_coils)
        self.reduction = int(reduction)
        self.reduced = tuple(g // reduction for g in self.grid)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        flags = (B.PISCO_FLAG_HOST_IO if host_io else 0) | precision_flags(precision)
        if masked_gram:
            flags |= B.PISCO_FLAG_MASKED_GRAM
        if block_pi:
            flags |= B.PISCO_FLAG_BLOCK_PI
        if gram_df:
            flags |= B.PISCO_FLAG_GRAM_DF
        if tc_interp:
            flags |= B.PISCO_FLAG_TC_INTERP
        if g_dense:
            flags |= B.PISCO_FLAG_G_DENSE
        self.params = B.make_params(self.grid, self.calib_shape, self.Q, tau, kernel_shape, thr,
                                    reduction, iters, seed, flags, eig_block, eig_iters, tc_splits,
                                    gemm_splits, gemm_tile)
        st, h = B.pisco_plan(self.params, self.stream.cuda_stream)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_plan")
        self._plan = h
        self.last_status = None

    # ------------------------------------------------------------------------------------
    def estimate_into(self, calib: torch.Tensor, maps: torch.Tensor, eig: torch.Tensor | None):
        """Run on device tensors (complex64 calib [Q,*calib], maps [Q,*grid], float32 eig)."""
        for t, name in ((calib, "calib"), (maps, "maps")):
            if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex64 CUDA tensor")
        if tuple(calib.shape) != (self.Q,) + self.calib_shape:
            raise ValueError(f"calib shape {tuple(calib.shape)} != {(self.Q,) + self.calib_shape}")
        if tuple(maps.shape) != (self.Q,) + self.grid:
            raise ValueError(f"maps shape {tuple(maps.shape)} != {(self.Q,) + self.grid}")
        if eig is not None and (eig.dtype != torch.float32 or not eig.is_cuda or eig.numel() != int(np.prod(self.reduced))):
            raise ValueError("eig must be a float32 CUDA tensor with one entry per reduced pixel")
        st = B.pisco_estimate(self._plan, calib.data_ptr(), maps.data_ptr(),
                              eig.data_ptr() if eig is not None else None)
        self.last_status = st
        if st not in (B.PISCO_OK, B.PISCO_ERR_RANK):
            raise B.PiscoError(st, "pisco_estimate")
        return st

    def __call__(self, calib: torch.Tensor):
        maps = torch.empty((self.Q,) + self.grid, dtype=torch.complex64, device=calib.device)
        eig = torch.empty(self.reduced, dtype=torch.float32, device=calib.device)
        self.estimate_into(calib.contiguous(), maps, eig)
        return maps, eig

    def estimate_host(self, calib: np.ndarray, maps: np.ndarray, eig: np.ndarray | None):
        """Host-buffer call (pisco_estimate_host): numpy complex64 in, numpy out."""
        if calib.dtype != np.complex64 or maps.dtype != np.complex64:
            raise ValueError("host buffers must be complex64")
        if not (calib.flags.c_contiguous and maps.flags.c_contiguous):
            raise ValueError("host buffers must be C-contiguous")
        st = B.pisco_estimate_host(self._plan, calib.ctypes.data, maps.ctypes.data,
                                   eig.ctypes.data if eig is not None else None)
        self.last_status = st
        if st not in (B.PISCO_OK, B.PISCO_ERR_RANK):
            raise B.PiscoError(st, "pisco_estimate_host")
        return st

    # ------------------------------------------------------------------------------------
    def info(self):
        st, R, k, ws = B.pisco_plan_info(self._plan)
        return dict(R=R, k=k, workspace_bytes=ws)

    def stats(self):
        st, d = B.pisco_get_stats(self._plan)
        return d

    def set_profiling(self, enable=True):
        B.pisco_set_profiling(self._plan, enable)

    def profile_reset(self):
        B.pisco_profile_reset(self._plan)

    def profile(self):
        return B.pisco_profile(self._plan)

    _BUF_TYPES = {B.PISCO_BUF_LAGS: "<c16", B.PISCO_BUF_GRAM: "<c16", B.PISCO_BUF_SIGNAL: "<c8",
                  B.PISCO_BUF_WEIGHTS: "<f4", B.PISCO_BUF_RITZ: "<f8", B.PISCO_BUF_G: "<c8",
                  B.PISCO_BUF_V: "<c8", B.PISCO_BUF_Y: "<c8", B.PISCO_BUF_BLOCK: "<c8",
                  B.PISCO_BUF_RITZ32: "<f4", B.PISCO_BUF_SCALE: "<f8"}

    def debug_buffer(self, which: int) -> torch.Tensor:
        """A copy of one intermediate buffer of the last estimate (flat tensor)."""
        st, ptr, nbytes = B.pisco_debug_buffer(self._plan, which)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_debug_buffer")
        ts = self._BUF_TYPES[which]
        item = int(ts[2:])
        view = _DevView(ptr, (nbytes // item,), ts)
        self.stream.synchronize()
        return torch.as_tensor(view, device="cuda").clone()

    def support_mask(self, eig: torch.Tensor, threshold=0.05) -> torch.Tensor:
        """uint8 mask of the reduced-grid pixels with eigenvalue below threshold (inside the object)."""
        mask = torch.empty(eig.shape, dtype=torch.uint8, device=eig.device)
        st = B.pisco_support_mask(eig.data_ptr(), eig.numel(), threshold, mask.data_ptr(), self.stream.cuda_stream)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_support_mask")
        return mask

    def close(self):
        if getattr(self, "_plan", None):
            B.pisco_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PiscoBatch:
    """A batch of independent estimates (shapes may differ), run as one CUDA graph.

    specs: list of dicts with keys grid, calib_shape, num_coils, tau and optionally
    kernel_shape, thr, reduction, iters, seed, eig_block, eig_iters, precision, tc_splits,
    gemm_splits, gemm_tile, gram_df, tc_interp, batch_group (items of identical parameters
    estimated by one batched pass; 0 automatic, 1 one launch chain per item).
    """

    def __init__(self, specs, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("PiscoBatch needs a CUDA GPU (no CPU fallback)")
        self.specs = [dict(s) for s in specs]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        params = []
        for sp in self.specs:
            params.append(B.make_params(tuple(sp["grid"]), tuple(sp["calib_shape"]), sp["num_coils"],
                                        sp["tau"], sp.get("kernel_shape", "ellipsoid"),
                                        sp.get("thr", 0.05), sp.get("reduction", 1),
                                        sp.get("iters", 30), sp.get("seed", 0),
                                        precision_flags(sp.get("precision", "fp32"))
                                        | (B.PISCO_FLAG_GRAM_DF if sp.get("gram_df") else 0)
                                        | (B.PISCO_FLAG_TC_INTERP if sp.get("tc_interp") else 0),
                                        sp.get("eig_block", 0), sp.get("eig_iters", 0), sp.get("tc_splits", 0),
                                        sp.get("gemm_splits", 0), sp.get("gemm_tile", 0),
                                        sp.get("batch_group", 0)))
        st, h = B.pisco_batch_plan(params, self.stream.cuda_stream)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_batch_plan")
        self._b = h
        self.last_item_status = None

    def __len__(self):
        return len(self.specs)

    def estimate_into(self, calibs, maps, eigs=None):
        st, items = B.pisco_batch_estimate(self._b, [c.data_ptr() for c in calibs],
                                           [m.data_ptr() for m in maps],
                                           [e.data_ptr() if e is not None else 0 for e in eigs] if eigs is not None else None)
        self.last_item_status = items
        if st not in (B.PISCO_OK, B.PISCO_ERR_RANK):
            raise B.PiscoError(st, "pisco_batch_estimate")
        return st

    def estimate_host(self, calibs, maps, eigs=None):
        st, items = B.pisco_batch_estimate(self._b, [c.ctypes.data for c in calibs],
                                           [m.ctypes.data for m in maps],
                                           [e.ctypes.data for e in eigs] if eigs is not None else None,
                                           host=True)
        self.last_item_status = items
        if st not in (B.PISCO_OK, B.PISCO_ERR_RANK):
            raise B.PiscoError(st, "pisco_batch_estimate_host")
        return st

    def launch(self, calibs, maps, eigs=None):
        """Enqueue a device-buffer call (after the work on the batch's stream, which then waits for
        it) and return at once; wait() decodes the statuses.  Two batch objects launched in turn
        keep the GPU busy while the host prepares the next launch."""
        st = B.pisco_batch_launch(self._b, [c.data_ptr() for c in calibs], [m.data_ptr() for m in maps],
                                  [e.data_ptr() if e is not None else 0 for e in eigs] if eigs is not None else None)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_batch_launch")

    def launch_host(self, calibs, maps, eigs=None):
        """Enqueue a host-buffer call and return at once (pinned numpy buffers that stay untouched
        until wait()); two batch objects can then overlap one step's copies with the next step."""
        st = B.pisco_batch_launch_host(self._b, [c.ctypes.data for c in calibs], [m.ctypes.data for m in maps],
                                       [e.ctypes.data for e in eigs] if eigs is not None else None)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_batch_launch_host")

    def wait(self):
        st, items = B.pisco_batch_wait(self._b, len(self.specs))
        self.last_item_status = items
        if st not in (B.PISCO_OK, B.PISCO_ERR_RANK):
            raise B.PiscoError(st, "pisco_batch_wait")
        return st

    def alloc_outputs(self, device="cuda"):
        maps, eigs = [], []
        for sp in self.specs:
            g = tuple(sp["grid"])
            r = tuple(x // sp.get("reduction", 1) for x in g)
            maps.append(torch.empty((sp["num_coils"],) + g, dtype=torch.complex64, device=device))
            eigs.append(torch.empty(r, dtype=torch.float32, device=device))
        return maps, eigs

    def info(self):
        st, c, l, w = B.pisco_batch_info(self._b)
        return dict(count=c, launches=l, workspace_bytes=w)

    def debug_buffer(self, i, which: int) -> torch.Tensor:
        """A copy of one intermediate buffer of item i's last estimate (flat tensor)."""
        st, h = B.pisco_batch_item(self._b, i)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_batch_item")
        st, ptr, nbytes = B.pisco_debug_buffer(h, which)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_debug_buffer")
        ts = PiscoEstimator._BUF_TYPES[which]
        view = _DevView(ptr, (nbytes // int(ts[2:]),), ts)
        torch.cuda.synchronize()
        return torch.as_tensor(view, device="cuda").clone()

    def set_profiling(self, enable=True):
        """Eager calls with CUDA events around every operation of every group's pass."""
        st = B.pisco_batch_set_profiling(self._b, enable)
        if st != B.PISCO_OK:
            raise B.PiscoError(st, "pisco_batch_set_profiling")

    def profile_reset(self):
        B.pisco_batch_profile_reset(self._b)

    def profile(self):
        """{operation: (total_ms, count)} summed over the groups since the last reset."""
        return B.pisco_batch_profile(self._b)

    def groups(self):
        st, g, mx = B.pisco_batch_groups(self._b)
        return dict(groups=g, largest=mx)

    def item_stats(self, i):
        st, h = B.pisco_batch_item(self._b, i)
        return B.pisco_get_stats(h)[1]

    def close(self):
        if getattr(self, "_b", None):
            B.pisco_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
