"""The C-ABI library loads and exports every function include/vdwgb.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vdwgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vdwgb_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_06999_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_paper_shaped_calls():
    names = _declared()
    for n in ("vdwgb_new", "vdwgb_set_unit_cell", "vdwgb_init_cuda", "vdwgb_calculate",
              "vdwgb_calculate_device", "vdwgb_finalize"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1703_06999_gb300 import binding
    for n in _declared():
        assert hasattr(binding, n), n


def test_host_side_validation_without_gpu():
    from paper_1703_06999_gb300 import binding as B
    h = B.vdwgb_new(B.DF2)
    try:
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_set_unit_cell(h, (11, 4, 4), [[1, 0, 0], [0, 1, 0], [0, 0, 1]])
        assert ei.value.code == -1
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_set_unit_cell(h, (4, 4, 4), [[1, 0, 0], [2, 0, 0], [0, 0, 1]])
        assert ei.value.code == -1
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_init_cuda(h, 0, B.FP64)
        assert ei.value.code == -4          # cell not set yet
    finally:
        B.vdwgb_finalize(h)
    with pytest.raises(B.VdwgbError):
        B.vdwgb_new(3)
    assert B.vdwgb_footprint_bytes((96, 96, 96), B.FP32_MIXED) < B.vdwgb_footprint_bytes((96, 96, 96), B.FP64)


def test_fault_injection_arguments_without_gpu():
    from paper_1703_06999_gb300 import binding as B
    B.vdwgb_inject_fault(B.FAULT_ALLOC, 2)
    B.vdwgb_inject_fault(B.FAULT_NONE, 0)                # disarms
    for kind, count in ((7, 1), (B.FAULT_WAIT, -1)):
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_inject_fault(kind, count)
        assert ei.value.code == -1


def test_kernel_table_argument_checks_without_gpu():
    import numpy as np
    from paper_1703_06999_gb300 import binding as B
    h = B.vdwgb_new(B.DF1)
    try:
        tab = np.zeros((210, 1024))
        B.vdwgb_set_kernel_k(h, tab)                   # accepted before init
        tab[3, 7] = np.nan
        with pytest.raises(B.VdwgbError) as ei:
            B.vdwgb_set_kernel_k(h, tab)
        assert ei.value.code == -1
        B.vdwgb_set_kernel_k(h, None)                  # back to the vdW-DF table
        with pytest.raises(ValueError):
            B.vdwgb_set_kernel_k(h, np.zeros(10))
    finally:
        B.vdwgb_finalize(h)
