"""ctypes binding of the C ABI declared in include/pisco.h (argument marshalling only).

Every computation happens in the CUDA library; this module converts Python/torch arguments
to the plain pointers and sizes the ABI takes.  Importing it loads `_lib/libpisco.so` and
raises if the library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libpisco.so")

PISCO_OK, PISCO_ERR_ARG, PISCO_ERR_CUDA, PISCO_ERR_OOM, PISCO_ERR_RANK, PISCO_ERR_TIMEOUT, \
    PISCO_ERR_NOT_CONVERGED, PISCO_ERR_UNSUPPORTED, PISCO_ERR_TOO_LARGE = range(9)
PISCO_KERNEL_RECT, PISCO_KERNEL_ELLIPSOID = 0, 1
PISCO_FLAG_HOST_IO = 0x1
PISCO_FLAG_TC_GFIELD = 0x2
PISCO_FLAG_TC_EIG = 0x4
PISCO_FLAG_TC_1PASS = 0x8
PISCO_FLAG_MASKED_GRAM = 0x10
PISCO_FLAG_BLOCK_PI = 0x20
PISCO_FLAG_GRAM_DF = 0x40
PISCO_FLAG_TC_THIN = 0x80
PISCO_FLAG_TC_INTERP = 0x100
PISCO_FLAG_G_DENSE = 0x200
(PISCO_BUF_LAGS, PISCO_BUF_GRAM, PISCO_BUF_SIGNAL, PISCO_BUF_WEIGHTS, PISCO_BUF_RITZ, PISCO_BUF_G,
 PISCO_BUF_V, PISCO_BUF_Y, PISCO_BUF_BLOCK, PISCO_BUF_RITZ32, PISCO_BUF_SCALE) = range(11)


class pisco_params(ctypes.Structure):
    _fields_ = [
        ("ndim", ctypes.c_int),
        ("grid", ctypes.c_int * 3),
        ("calib", ctypes.c_int * 3),
        ("num_coils", ctypes.c_int),
        ("kernel_shape", ctypes.c_int),
        ("kernel_radius", ctypes.c_int * 3),
        ("null_threshold", ctypes.c_double),
        ("grid_reduction", ctypes.c_int),
        ("power_iters", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
        ("flags", ctypes.c_uint),
        ("eig_block", ctypes.c_int),
        ("eig_iters", ctypes.c_int),
        ("tc_splits", ctypes.c_int),
        ("gemm_splits", ctypes.c_int),
        ("gemm_tile", ctypes.c_int),
        ("batch_group", ctypes.c_int),
    ]


class pisco_stats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int),
        ("eig_block", ctypes.c_int),
        ("eig_iters", ctypes.c_int),
        ("jacobi_sweeps", ctypes.c_int),
        ("nband", ctypes.c_int),
        ("lambda_max", ctypes.c_double),
        ("signal_dim", ctypes.c_int),
        ("filter_len", ctypes.c_int),
        ("warm_fallback", ctypes.c_int),
        ("cert_margin", ctypes.c_double),
        ("band_resid", ctypes.c_double),
    ]


class PiscoError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {pisco_status_string(status)} (status {status})")


_lib = None


def load():
    """Load libpisco.so (built by build_ext.build()); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"PISCO CUDA library not found at {LIB_PATH}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.pisco_plan.argtypes = [P(pisco_params), vp, P(vp)]
    lib.pisco_plan.restype = ctypes.c_int
    lib.pisco_estimate.argtypes = [vp, vp, vp, vp]
    lib.pisco_estimate.restype = ctypes.c_int
    lib.pisco_estimate_host.argtypes = [vp, vp, vp, vp]
    lib.pisco_estimate_host.restype = ctypes.c_int
    lib.pisco_destroy.argtypes = [vp]
    lib.pisco_destroy.restype = None
    lib.pisco_status_string.argtypes = [ctypes.c_int]
    lib.pisco_status_string.restype = ctypes.c_char_p
    lib.pisco_plan_info.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_size_t)]
    lib.pisco_plan_info.restype = ctypes.c_int
    lib.pisco_debug_buffer.argtypes = [vp, ctypes.c_int, P(vp), P(ctypes.c_size_t)]
    lib.pisco_debug_buffer.restype = ctypes.c_int
    lib.pisco_get_stats.argtypes = [vp, P(pisco_stats)]
    lib.pisco_get_stats.restype = ctypes.c_int
    lib.pisco_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.pisco_set_profiling.restype = ctypes.c_int
    lib.pisco_profile_reset.argtypes = [vp]
    lib.pisco_profile_reset.restype = ctypes.c_int
    lib.pisco_profile_entry.argtypes = [vp, ctypes.c_int, P(ctypes.c_char_p), P(ctypes.c_double),
                                        P(ctypes.c_int)]
    lib.pisco_profile_entry.restype = ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.pisco_batch_plan.argtypes = [P(pisco_params), ctypes.c_int, vp, P(vp)]
    lib.pisco_batch_plan.restype = ctypes.c_int
    lib.pisco_batch_estimate.argtypes = [vp, PP, PP, PP, P(ctypes.c_int)]
    lib.pisco_batch_estimate.restype = ctypes.c_int
    lib.pisco_batch_estimate_host.argtypes = [vp, PP, PP, PP, P(ctypes.c_int)]
    lib.pisco_batch_estimate_host.restype = ctypes.c_int
    lib.pisco_batch_launch_host.argtypes = [vp, PP, PP, PP]
    lib.pisco_batch_launch_host.restype = ctypes.c_int
    lib.pisco_batch_launch.argtypes = [vp, PP, PP, PP]
    lib.pisco_batch_launch.restype = ctypes.c_int
    lib.pisco_batch_wait.argtypes = [vp, P(ctypes.c_int)]
    lib.pisco_batch_wait.restype = ctypes.c_int
    lib.pisco_batch_info.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_size_t)]
    lib.pisco_batch_info.restype = ctypes.c_int
    lib.pisco_batch_item.argtypes = [vp, ctypes.c_int, P(vp)]
    lib.pisco_batch_item.restype = ctypes.c_int
    lib.pisco_test_stall_tensor_loads.argtypes = [ctypes.c_int]
    lib.pisco_test_stall_tensor_loads.restype = None
    lib.pisco_batch_set_profiling.argtypes = [vp, ctypes.c_int]
    lib.pisco_batch_set_profiling.restype = ctypes.c_int
    lib.pisco_batch_profile_reset.argtypes = [vp]
    lib.pisco_batch_profile_reset.restype = ctypes.c_int
    lib.pisco_batch_profile_entry.argtypes = [vp, ctypes.c_int, P(ctypes.c_char_p), P(ctypes.c_double),
                                              P(ctypes.c_int)]
    lib.pisco_batch_profile_entry.restype = ctypes.c_int
    lib.pisco_batch_groups.argtypes = [vp, P(ctypes.c_int), P(ctypes.c_int)]
    lib.pisco_batch_groups.restype = ctypes.c_int
    lib.pisco_batch_destroy.argtypes = [vp]
    lib.pisco_batch_destroy.restype = None
    lib.pisco_gram_lags_noalloc.argtypes = [P(pisco_params), vp, vp, vp]
    lib.pisco_gram_lags_noalloc.restype = ctypes.c_int
    lib.pisco_tc_cgemm_pipelined_workspace.argtypes = [ctypes.c_int] * 5
    lib.pisco_tc_cgemm_pipelined_workspace.restype = ctypes.c_size_t
    lib.pisco_tc_cgemm_pipelined.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             P(ctypes.c_float), vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int,
                                             P(ctypes.c_float), vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t,
                                             vp, vp]
    lib.pisco_tc_cgemm_pipelined.restype = ctypes.c_int
    fp = P(ctypes.c_float)
    lib.pisco_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, fp, ctypes.c_longlong, vp, P(vp)]
    lib.pisco_mlp_create.restype = ctypes.c_int
    lib.pisco_mlp_write.argtypes = [vp, fp]
    lib.pisco_mlp_write.restype = ctypes.c_int
    lib.pisco_mlp_forward.argtypes = [vp, vp, ctypes.c_longlong, vp]
    lib.pisco_mlp_forward.restype = ctypes.c_int
    lib.pisco_mlp_backward.argtypes = [vp, vp, vp, ctypes.c_longlong, P(ctypes.c_double)]
    lib.pisco_mlp_backward.restype = ctypes.c_int
    lib.pisco_mlp_adam.argtypes = [vp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    lib.pisco_mlp_adam.restype = ctypes.c_int
    lib.pisco_mlp_read.argtypes = [vp, ctypes.c_int, fp]
    lib.pisco_mlp_read.restype = ctypes.c_int
    lib.pisco_mlp_destroy.argtypes = [vp]
    lib.pisco_mlp_destroy.restype = None
    lib.pisco_support_mask.argtypes = [vp, ctypes.c_longlong, ctypes.c_float, vp, vp]
    lib.pisco_support_mask.restype = ctypes.c_int
    lib.pisco_set_warm_start.argtypes = [vp, vp, ctypes.c_int, ctypes.c_float, ctypes.c_int]
    lib.pisco_set_warm_start.restype = ctypes.c_int
    lib.pisco_warm_start_features.argtypes = [vp, ctypes.c_int, ctypes.c_longlong, vp, vp]
    lib.pisco_warm_start_features.restype = ctypes.c_int
    lib.pisco_warm_start_patch_features.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                    ctypes.c_int, vp, vp]
    lib.pisco_warm_start_patch_features.restype = ctypes.c_int
    lib.pisco_mlp_set_loss.argtypes = [vp, ctypes.c_int]
    lib.pisco_mlp_set_loss.restype = ctypes.c_int
    _lib = lib
    return lib


def pisco_status_string(status: int) -> str:
    return load().pisco_status_string(int(status)).decode()


def make_params(grid, calib, num_coils, kernel_radius, kernel_shape="ellipsoid", null_threshold=0.05,
                grid_reduction=1, power_iters=30, seed=0, flags=0, eig_block=0, eig_iters=0, tc_splits=0,
                gemm_splits=0, gemm_tile=0, batch_group=0):
    """pisco_params from (z,)y,x-ordered Python tuples (the array order); the struct is x,y,z."""
    nd = len(grid)
    pr = pisco_params()
    pr.ndim = nd
    g = list(grid)[::-1] + [1] * (3 - nd)
    c = list(calib)[::-1] + [1] * (3 - nd)
    tau = list(kernel_radius if not isinstance(kernel_radius, int) else [kernel_radius] * nd)[::-1] + [0] * (3 - nd)
    for d in range(3):
        pr.grid[d], pr.calib[d], pr.kernel_radius[d] = g[d], c[d], tau[d]
    pr.num_coils = num_coils
    pr.kernel_shape = {"rect": PISCO_KERNEL_RECT, "ellipsoid": PISCO_KERNEL_ELLIPSOID}[kernel_shape]
    pr.null_threshold = null_threshold
    pr.grid_reduction = grid_reduction
    pr.power_iters = power_iters
    pr.seed = seed
    pr.flags = flags
    pr.eig_block = eig_block
    pr.eig_iters = eig_iters
    pr.tc_splits = tc_splits
    pr.gemm_splits = gemm_splits
    pr.gemm_tile = gemm_tile
    pr.batch_group = batch_group
    return pr


def pisco_plan(params: pisco_params, stream: int = 0):
    """Returns (status, plan handle)."""
    h = ctypes.c_void_p()
    st = load().pisco_plan(ctypes.byref(params), ctypes.c_void_p(stream), ctypes.byref(h))
    return st, h


def pisco_estimate(plan, d_calib: int, d_maps: int, d_eig: int | None):
    return load().pisco_estimate(plan, ctypes.c_void_p(d_calib), ctypes.c_void_p(d_maps),
                                 ctypes.c_void_p(d_eig or 0))


def pisco_estimate_host(plan, h_calib: int, h_maps: int, h_eig: int | None):
    return load().pisco_estimate_host(plan, ctypes.c_void_p(h_calib), ctypes.c_void_p(h_maps),
                                      ctypes.c_void_p(h_eig or 0))


def pisco_destroy(plan):
    load().pisco_destroy(plan)


def pisco_plan_info(plan):
    R, k, ws = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    st = load().pisco_plan_info(plan, ctypes.byref(R), ctypes.byref(k), ctypes.byref(ws))
    return st, R.value, k.value, ws.value


def pisco_debug_buffer(plan, which: int):
    p, nb = ctypes.c_void_p(), ctypes.c_size_t()
    st = load().pisco_debug_buffer(plan, int(which), ctypes.byref(p), ctypes.byref(nb))
    return st, p.value, nb.value


def pisco_get_stats(plan):
    st = pisco_stats()
    rc = load().pisco_get_stats(plan, ctypes.byref(st))
    return rc, {f: getattr(st, f) for f, _ in pisco_stats._fields_}


def pisco_set_profiling(plan, enable: bool):
    return load().pisco_set_profiling(plan, 1 if enable else 0)


def pisco_profile_reset(plan):
    return load().pisco_profile_reset(plan)


def pisco_profile(plan):
    """{name: (total_ms, count)} accumulated since profiling was enabled or reset."""
    out = {}
    i = 0
    name, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int()
    while load().pisco_profile_entry(plan, i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt)) == PISCO_OK:
        out[name.value.decode()] = (ms.value, cnt.value)
        i += 1
    return out


def pisco_gram_lags_noalloc(params: pisco_params, d_calib: int, d_lags: int, stream: int = 0):
    """Allocation-free lag-table entry point (see include/pisco.h)."""
    return load().pisco_gram_lags_noalloc(ctypes.byref(params), ctypes.c_void_p(d_calib),
                                          ctypes.c_void_p(d_lags), ctypes.c_void_p(stream))


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p if p else None
    return arr


def pisco_batch_plan(params_list, stream: int = 0):
    arr = (pisco_params * len(params_list))(*params_list)
    h = ctypes.c_void_p()
    st = load().pisco_batch_plan(arr, len(params_list), ctypes.c_void_p(stream), ctypes.byref(h))
    return st, h


def pisco_batch_estimate(batch, calibs, maps, eigs, host=False):
    n = len(calibs)
    stat = (ctypes.c_int * n)()
    fn = load().pisco_batch_estimate_host if host else load().pisco_batch_estimate
    st = fn(batch, _ptr_array(calibs), _ptr_array(maps), _ptr_array(eigs) if eigs is not None else None, stat)
    return st, list(stat)


def pisco_batch_launch_host(batch, calibs, maps, eigs):
    """Enqueue a host-buffer batch call; the pointer arrays are kept alive by the caller."""
    return load().pisco_batch_launch_host(batch, _ptr_array(calibs), _ptr_array(maps),
                                          _ptr_array(eigs) if eigs is not None else None)


def pisco_batch_launch(batch, calibs, maps, eigs):
    """Enqueue a device-buffer batch call (ordered on the batch's caller stream)."""
    return load().pisco_batch_launch(batch, _ptr_array(calibs), _ptr_array(maps),
                                     _ptr_array(eigs) if eigs is not None else None)


def pisco_batch_wait(batch, n):
    stat = (ctypes.c_int * n)()
    st = load().pisco_batch_wait(batch, stat)
    return st, list(stat)


def pisco_batch_info(batch):
    c, l, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t()
    st = load().pisco_batch_info(batch, ctypes.byref(c), ctypes.byref(l), ctypes.byref(w))
    return st, c.value, l.value, w.value


def pisco_test_stall_tensor_loads(enable: bool):
    """Test hook: tensor-core products withhold their loads so their bounded waits expire."""
    load().pisco_test_stall_tensor_loads(1 if enable else 0)


def pisco_batch_set_profiling(batch, enable: bool):
    return load().pisco_batch_set_profiling(batch, 1 if enable else 0)


def pisco_batch_profile_reset(batch):
    return load().pisco_batch_profile_reset(batch)


def pisco_batch_profile(batch):
    """{name: (total_ms, count)} of the batch's operations (summed over its groups)."""
    out = {}
    i = 0
    name, ms, cnt = ctypes.c_char_p(), ctypes.c_double(), ctypes.c_int()
    while load().pisco_batch_profile_entry(batch, i, ctypes.byref(name), ctypes.byref(ms), ctypes.byref(cnt)) == PISCO_OK:
        out[name.value.decode()] = (ms.value, cnt.value)
        i += 1
    return out


def pisco_batch_groups(batch):
    g, mx = ctypes.c_int(), ctypes.c_int()
    st = load().pisco_batch_groups(batch, ctypes.byref(g), ctypes.byref(mx))
    return st, g.value, mx.value


def pisco_batch_item(batch, i):
    h = ctypes.c_void_p()
    st = load().pisco_batch_item(batch, i, ctypes.byref(h))
    return st, h


def pisco_batch_destroy(batch):
    load().pisco_batch_destroy(batch)


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def pisco_mlp_create(n_in, n_hidden, n_out, params, max_batch, stream=0):
    """params: float32 numpy blob [W1|b1|W2|b2|W3|b3].  Returns (status, handle)."""
    import numpy as np
    blob = np.ascontiguousarray(params, dtype=np.float32)
    h = ctypes.c_void_p()
    st = load().pisco_mlp_create(n_in, n_hidden, n_out, _fptr(blob), max_batch, ctypes.c_void_p(stream),
                                 ctypes.byref(h))
    return st, h


def pisco_mlp_write(mlp, params):
    import numpy as np
    blob = np.ascontiguousarray(params, dtype=np.float32)
    return load().pisco_mlp_write(mlp, _fptr(blob))


def pisco_mlp_forward(mlp, d_x, batch, d_out):
    return load().pisco_mlp_forward(mlp, ctypes.c_void_p(d_x), batch, ctypes.c_void_p(d_out))


def pisco_mlp_backward(mlp, d_x, d_t, batch, want_loss=True):
    """Returns (status, loss or None)."""
    loss = ctypes.c_double()
    st = load().pisco_mlp_backward(mlp, ctypes.c_void_p(d_x), ctypes.c_void_p(d_t), batch,
                                   ctypes.byref(loss) if want_loss else None)
    return st, (loss.value if want_loss else None)


def pisco_mlp_adam(mlp, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    return load().pisco_mlp_adam(mlp, lr, beta1, beta2, eps)


def pisco_mlp_read(mlp, which, nparam):
    import numpy as np
    out = np.empty(nparam, np.float32)
    st = load().pisco_mlp_read(mlp, which, _fptr(out))
    return st, out


def pisco_mlp_destroy(mlp):
    load().pisco_mlp_destroy(mlp)


def pisco_set_warm_start(plan, mlp, iters, gate, fallback_iters):
    return load().pisco_set_warm_start(plan, mlp, iters, gate, fallback_iters)


def pisco_warm_start_patch_features(d_y, Q, dims, radius, d_x, stream=0):
    d = (ctypes.c_int * 3)(*[int(v) for v in dims] + [0] * (3 - len(dims)))
    return load().pisco_warm_start_patch_features(ctypes.c_void_p(d_y), Q, d, len(dims), radius,
                                                  ctypes.c_void_p(d_x), ctypes.c_void_p(stream))


def pisco_mlp_set_loss(h, kind):
    return load().pisco_mlp_set_loss(h, int(kind))


def pisco_warm_start_features(d_y, Q, npix, d_x, stream=0):
    return load().pisco_warm_start_features(ctypes.c_void_p(d_y), Q, npix, ctypes.c_void_p(d_x),
                                            ctypes.c_void_p(stream))


def pisco_tc_cgemm_pipelined_workspace(nterms, M, N, K, splits):
    return load().pisco_tc_cgemm_pipelined_workspace(nterms, M, N, K, splits)


def pisco_tc_cgemm_pipelined(nterms, M, N, K, alpha, d_A, lda, d_B, ldb, opB, beta, d_C, ldc, splits, d_ws,
                             ws_bytes, d_status=0, stream=0):
    a = (ctypes.c_float * 2)(float(complex(alpha).real), float(complex(alpha).imag))
    b = (ctypes.c_float * 2)(float(complex(beta).real), float(complex(beta).imag))
    return load().pisco_tc_cgemm_pipelined(nterms, M, N, K, a, ctypes.c_void_p(d_A), lda, ctypes.c_void_p(d_B), ldb,
                                           opB, b, ctypes.c_void_p(d_C), ldc, splits, ctypes.c_void_p(d_ws),
                                           ws_bytes, ctypes.c_void_p(d_status or 0), ctypes.c_void_p(stream))


def pisco_support_mask(d_eig, n, threshold, d_mask, stream=0):
    return load().pisco_support_mask(ctypes.c_void_p(d_eig), n, threshold, ctypes.c_void_p(d_mask),
                                     ctypes.c_void_p(stream))

