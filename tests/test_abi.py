"""The C-ABI library builds, loads and exports every symbol of include/ptm.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ptm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ptm_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1603_05143_gb300 import build, load
    build.build()
    return load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ptm_create", "ptm_destroy", "ptm_classify_frame", "ptm_classify_frame_host",
              "ptm_get_stats", "ptm_status_string"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    for code, name in enumerate(("PTM_OK", "PTM_ERR_INVALID_ARG", "PTM_ERR_OUT_OF_MEMORY", "PTM_ERR_CUDA",
                                 "PTM_ERR_TIMEOUT", "PTM_ERR_DEVICE_STATUS", "PTM_ERR_BUSY", "PTM_ERR_NOT_FOUND")):
        assert lib.ptm_status_string(code).decode() == name
    assert lib.ptm_status_string(99).decode() == "PTM_ERR_UNKNOWN"


def test_null_arguments_rejected_without_gpu(lib):
    from paper_1603_05143_gb300.binding import ptm_frame, ptm_outputs
    assert lib.ptm_create(None, None) == 1
    assert lib.ptm_destroy(None) == 1
    assert lib.ptm_classify_frame(None, ctypes.byref(ptm_frame()), ctypes.byref(ptm_outputs()), None) == 1
    assert lib.ptm_get_stats(None, None) == 1
    assert lib.ptm_measure_fma_peak(2, None, None) == 1


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1603_05143_gb300 import PTM, PTMError
    with pytest.raises(PTMError):
        PTM(0)
