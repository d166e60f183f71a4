"""The C ABI library builds, loads and exports every symbol include/*.h declares (no GPU)."""
import glob
import os
import re

import pytest

from paper_2404_05708_gb300 import build, dfd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_in_headers():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:dfd_status|const char\s*\*|double)\s+(dfd_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dfd.load_library()


def test_header_declares_entry_points():
    names = declared_in_headers()
    for n in ("dfd_pair", "dfd_pair_reference", "dfd_context_create", "dfd_get_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_in_headers() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared_in_headers() <= set(dfd.declared_symbols())


def test_status_strings(lib):
    assert dfd.dfd_status_string(0) == "DFD_OK"
    assert dfd.dfd_status_string(6) == "DFD_ERR_TIMEOUT"
    for code, name in dfd.STATUS.items():
        assert dfd.dfd_status_string(code) == name


def test_options_default(lib):
    o = dfd.dfd_options_default()
    assert o.check_inputs == 1 and o.wait_timeout_ms == 2000.0


def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_cuda(), reason="checks the no-device path")
def test_no_cpu_fallback_without_device(lib):
    """Without a CUDA device the library refuses to compute (no CPU fallback)."""
    with pytest.raises(dfd.DFDError) as e:
        dfd.dfd_context_create(0)
    assert e.value.status == dfd.STATUS_CODE["DFD_ERR_CUDA"]


def test_entry_points_reject_null_context_without_touching_a_device(lib):
    """Host-side validation: every computing entry point returns
    DFD_ERR_INVALID_ARG for a NULL context before any CUDA call."""
    inv = dfd.STATUS_CODE["DFD_ERR_INVALID_ARG"]
    dummy = 0x1000   # never dereferenced: the NULL context is rejected first
    assert dfd.dfd_pair(None, dfd.DFD_F32, 2, dummy, 4, dummy, 4, dummy, dummy, None) == inv
    assert dfd.dfd_batch(None, dfd.DFD_F32, 2, dummy, dummy, 2, dummy, 1, dummy, dummy, None) == inv
    assert dfd.dfd_matrix(None, dfd.DFD_F32, 2, dummy, dummy, 3, dummy, dummy, None) == inv
    assert dfd.dfd_batch_decide(None, dfd.DFD_F32, 2, dummy, dummy, 2, dummy, 1, None, 1.0, dummy, dummy,
                                None, None) == inv
    assert dfd.dfd_knn(None, 2, dummy, 4, dummy, dummy, 2, None, 2, 1, dummy, dummy, None, None, None, None) == inv
    assert dfd.dfd_batch_variant(None, dfd.DFD_VARIANT_DTW, dfd.DFD_F32, 2, dummy, dummy, 2, dummy, 1, dummy,
                                 None) == inv
    assert dfd.dfd_mc_pair(None, 2, dummy, 4, dummy, 4, dummy, dummy, 0.1, 0.1, 1, dummy, dummy, None) == inv
