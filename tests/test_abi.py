"""The C-ABI library builds, loads and exports every entry point its header
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import os
import shutil

import pytest

import paper_2505_04556_gb300 as pm

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists(pm.LIB_PATH),
                                reason="nvcc not available to build the library")


@pytest.fixture(scope="module")
def lib():
    pm.build()
    return pm.load()


def test_header_declares_the_boundary():
    names = pm.exported_names()
    for required in ("permanova_create", "permanova_destroy", "permanova_last_error",
                     "permanova_sW", "permanova_sW_host", "permanova_test",
                     "permanova_permutations", "permanova_sync", "permanova_set_form",
                     "permanova_plan_form", "permanova_scratch_bytes"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(pm.LIB_PATH)
    for name in pm.exported_names():
        assert hasattr(raw, name), name


def test_null_context_is_rejected_without_a_gpu(lib):
    vp = ctypes.c_void_p
    rc = lib.permanova_sW(None, None, 10, 10, None, pm.LABEL_U8, 2, 1, None, None, None)
    assert rc == pm.EINVAL
    assert lib.permanova_set_form(None, pm.FORM_BRUTE) == pm.EINVAL
    assert lib.permanova_scratch_bytes(None, 0, 100, 2, 10) == 0
    res = pm.permanova_result()
    assert lib.permanova_test(None, None, 10, 10, None, 2, 10, 1, ctypes.byref(res), None,
                              None) == pm.EINVAL
    assert lib.permanova_create(0, 0, None) == pm.EINVAL
    lib.permanova_destroy(None)  # no-op
    assert isinstance(lib.permanova_last_error(vp()), bytes)


def test_label_type_codes_match_header():
    txt = open(pm.HEADER).read()
    assert "PERMANOVA_LABEL_I32 = 0" in txt and "PERMANOVA_LABEL_U16 = 1" in txt
    assert "PERMANOVA_LABEL_U8 = 2" in txt
    assert "PERMANOVA_FORM_GEMM = 3" in txt and "PERMANOVA_ETIMEOUT = 4" in txt
