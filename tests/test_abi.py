"""The C ABI library builds for sm_103a, loads, exports every function include/pisco.h
declares, and rejects invalid plans on the host before touching the GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_13431_gb300 import _binding, build_ext
    build_ext.build()
    return _binding.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "pisco.h")).read()
    return sorted(set(re.findall(r"^\s*(?:pisco_status|void|const char\*)\s+(pisco_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ("pisco_plan", "pisco_estimate", "pisco_destroy", "pisco_status_string",
              "pisco_plan_info", "pisco_estimate_host", "pisco_debug_buffer"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_2302_13431_gb300 import _binding as B
    assert B.pisco_status_string(B.PISCO_OK) == "ok"
    assert "R < Q-1" in B.pisco_status_string(B.PISCO_ERR_RANK)
    assert B.pisco_status_string(99) == "unknown status"


@pytest.mark.parametrize("bad", [
    dict(grid=(64, 64), calib=(4, 4), tau=2),           # Nc <= 2 tau
    dict(grid=(16, 16), calib=(24, 24), tau=2),         # Nc > N
    dict(grid=(64, 64), calib=(24, 24), tau=2, red=3),  # N not divisible by f
    dict(grid=(8, 8), calib=(8, 8), tau=2, red=2),      # N/f < 2 tau + 1
    dict(grid=(64, 64), calib=(24, 24), tau=2, thr=1.5),
    dict(grid=(64, 64), calib=(24, 24), tau=2, iters=0),
    dict(grid=(64, 64), calib=(24, 24), tau=2, Q=1),
    dict(grid=(64, 64), calib=(24, 24), tau=2, Q=65),
    dict(grid=(64, 64), calib=(24, 24), tau=2, eig_block=7),
])
def test_invalid_plans_rejected_on_host(lib, bad):
    from paper_2302_13431_gb300 import _binding as B
    pr = B.make_params(bad["grid"], bad["calib"], bad.get("Q", 4), bad["tau"], "rect",
                       bad.get("thr", 0.05), bad.get("red", 1), bad.get("iters", 10),
                       eig_block=bad.get("eig_block", 0))
    st, h = B.pisco_plan(pr)
    assert st == B.PISCO_ERR_ARG
    assert not h.value


def test_null_arguments(lib):
    from paper_2302_13431_gb300 import _binding as B
    import ctypes
    assert lib.pisco_plan(None, None, None) == B.PISCO_ERR_ARG
    assert lib.pisco_estimate(None, None, None, None) == B.PISCO_ERR_ARG
    lib.pisco_destroy(None)
    assert lib.pisco_plan_info(None, None, None, None) == B.PISCO_ERR_ARG
    p, n = ctypes.c_void_p(), ctypes.c_size_t()
    assert lib.pisco_debug_buffer(None, 0, ctypes.byref(p), ctypes.byref(n)) == B.PISCO_ERR_ARG
