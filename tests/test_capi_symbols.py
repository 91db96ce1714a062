"""The C-ABI library builds, loads and exports every symbol include/lgf.h declares.

No compute call is made here (this file runs on machines without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from conftest import build_lib
    build_lib()
    from paper_1604_01814_gb300 import _binding
    return _binding.load()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "lgf.h")).read()
    return sorted(set(re.findall(r"LGF_API\s+[\w\s\*]*?\b(lgf_\w+)\s*\(", hdr)))


def test_header_declares_the_entry_points():
    names = declared_symbols()
    for n in ("lgf_table_build", "lgf_poisson_apply", "lgf_intfactor_apply", "lgf_batch_apply"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1604_01814_gb300 import _binding
    names = declared_symbols()
    assert sorted(names) == sorted(_binding.EXPORTS)
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings_and_version(lib):
    assert lib.lgf_version() == 10000
    for s in range(7):
        assert lib.lgf_status_string(s)
    assert b"table" in lib.lgf_status_string(6)


def test_struct_layouts_match_header():
    from paper_1604_01814_gb300 import _binding as b
    assert ctypes.sizeof(b.lgf_blockset) == 16
    assert ctypes.sizeof(b.lgf_options) == 8 + 4 * 4 + 16
    assert ctypes.sizeof(b.lgf_problem) == 2 * 16 + 2 * 8 + 4 * 4 + 2 * 8
    assert ctypes.sizeof(b.lgf_kernel_stat) == 48 + 8 + 8
    assert ctypes.sizeof(b.lgf_stats) == 16 * 8
    assert ctypes.sizeof(b.lgf_tune_info) == 11 * 8 + 8 + 4 * 8
    assert ctypes.sizeof(b.lgf_stage) == 16 + 8 + 9 * 8 + 2 * 8 + 4 * 4


def test_null_arguments_rejected_without_gpu(lib):
    # argument checks run before any CUDA call
    assert lib.lgf_ctx_create(None, None) == 1          # LGF_EINVAL
    assert lib.lgf_ctx_destroy(None) == 1
    assert lib.lgf_poisson_apply(None, None, None, None, None, 1, 1, 1.0, None) == 1
    assert lib.lgf_table_info(None, None, None) == 1


def test_context_creation_reports_missing_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.lgf_ctx_create(ctypes.byref(h), None) == 3   # LGF_ECUDA, no crash
