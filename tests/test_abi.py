"""The C-ABI library loads and exports every entry point declared in include/hm.h (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "hm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2209_10241_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "hm_build" in names and "hm_count_exact" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2209_10241_gb300 import binding
    assert sorted(binding.EXPORTS) == _declared()


def test_host_only_queries(lib):
    lib.hm_num_classes.restype = ctypes.c_int
    assert lib.hm_num_classes(3) == 6
    assert lib.hm_num_classes(4) == 171
    assert lib.hm_num_classes(2) == -1
    cls = ctypes.c_int32()
    lib.hm_class_of_mask.restype = ctypes.c_int
    assert lib.hm_class_of_mask(4, 0b111111, ctypes.byref(cls)) == 0
    import oracle
    assert cls.value == oracle.class_of(4, 0b111111)
    assert lib.hm_class_of_mask(4, 1 << 11, ctypes.byref(cls)) == 1  # HM_EINVAL
