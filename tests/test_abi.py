"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/hj.h declares.  No kernel runs here (CPU only)."""
import ctypes
import os
import re

import pytest

from paper_1307_1955_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(hj_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(B.build())


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("hj_create", "hj_destroy", "hj_build", "hj_probe", "hj_partition", "hj_join", "hj_result_free",
                 "hj_sync", "hj_last_error"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_null_context_is_rejected_without_a_gpu(lib):
    lib.hj_join.restype = ctypes.c_int32
    assert lib.hj_join(None, None, None, None, None) == 1  # HJ_E_INVALID
    lib.hj_last_error.restype = ctypes.c_char_p
    assert lib.hj_last_error(None) == b"null context"


def test_profiling_calls_reject_a_null_context_without_a_gpu(lib):
    for name, args in (("hj_prof_enable", (None, 1)), ("hj_prof_only", (None, b"partition_join")),
                       ("hj_prof_only", (None, None)), ("hj_prof_reset", (None,)),
                       ("hj_prof_read", (None, None, 0, None))):
        f = getattr(lib, name)
        f.restype = ctypes.c_int32
        assert f(*args) == 1, name  # HJ_E_INVALID


def test_debug_hooks_reject_a_null_context_without_a_gpu(lib):
    for name, args in (("hj_debug_wait_limit", (None, ctypes.c_uint64(5))), ("hj_debug_scatter", (None, 0)),
                       ("hj_debug_scatter", (None, 2)), ("hj_debug_fail_alloc", (None, ctypes.c_int64(1)))):
        f = getattr(lib, name)
        f.restype = ctypes.c_int32
        assert f(*args) == 1, name  # HJ_E_INVALID


def test_server_calls_reject_null_handles_without_a_gpu(lib):
    for name, args in (("hj_server_create", (None, None, None)), ("hj_server_submit", (None, None, None, 0, None)),
                       ("hj_server_poll", (None, 1, None, None)), ("hj_server_destroy", (None,)),
                       ("hj_server_result_free", (None, None))):
        f = getattr(lib, name)
        f.restype = ctypes.c_int32
        assert f(*args) == 1, name  # HJ_E_INVALID


def test_binding_names_match_the_abi():
    from paper_1307_1955_gb300 import hj

    for name in ("hj_create", "hj_destroy", "hj_build", "hj_probe", "hj_table_free", "hj_partition", "hj_join",
                 "hj_result_free", "hj_sync", "hj_join_batch", "hj_server_create", "hj_server_submit",
                 "hj_server_poll", "hj_server_wait", "hj_server_result_free", "hj_server_destroy"):
        assert callable(getattr(hj, name))


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_1307_1955_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "hj_oracle" not in txt, f


def test_static_join_pair_buffer_is_checked_before_any_call():
    # A caller-owned pair buffer of the wrong shape, dtype, layout or device would
    # let the probe write past its end: the binding rejects it on the host.
    import torch

    from paper_1307_1955_gb300 import hj

    R = torch.zeros((4, 2), dtype=torch.int64)
    assert hj.check_pairs_buffer(None, R) == 0
    bad = [torch.zeros(8, dtype=torch.int64),                      # 1-D
           torch.zeros((4, 3), dtype=torch.int64),                 # three columns
           torch.zeros((4, 2), dtype=torch.int32),                 # narrower than R
           torch.zeros((2, 4), dtype=torch.int64).t(),             # not contiguous
           torch.zeros((4, 2), dtype=torch.int64),                 # host memory
           [[0, 0]]]                                               # not a tensor
    for p in bad:
        with pytest.raises(ValueError):
            hj.check_pairs_buffer(p, R)
    with pytest.raises(ValueError):                                # host relations
        hj.hj_join_static(R, R, None)
