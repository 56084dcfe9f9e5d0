"""The C ABI: libd8.so builds for sm_103a, loads without a GPU, exports every
function include/d8.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "d8.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w]+\s*\*?\s*(d8_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1605_05773_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 16, names
    for n in names:
        assert hasattr(lib, n), n


def test_host_side_errors_need_no_gpu(lib):
    vp = ctypes.c_void_p
    lib.d8_status_string.restype = ctypes.c_char_p
    lib.d8_stage_name.restype = ctypes.c_char_p
    lib.d8_version.restype = ctypes.c_char_p
    assert lib.d8_status_string(0) == b"ok"
    assert b"cycle" in lib.d8_status_string(4)
    assert lib.d8_stage_name(1) == b"tile_up"
    assert b"sm_103a" in lib.d8_version()
    assert lib.d8_create(None, 0) == 1  # D8_ERR_ARG
    assert lib.d8_set_tile(None, 64) == 1
    assert lib.d8_flowdir(None, None, 4, 4, 4, None, 4, 0, None) == 1
    assert lib.d8_accumulate(None, None, 4, 4, 4, None, 4, None) == 1
    assert lib.d8_get_status(None, None) == 1
    assert lib.d8_destroy(None) == 0
    assert lib.d8_batch_destroy(None) == 0
    assert lib.d8_set_strategy(None, 0) == 1
    assert lib.d8_fill(None, None, 4, 4, 4, ctypes.c_float(1e-3), None, 4, None, None) == 1
    assert lib.d8_combine_stats(None, None, None, 4) == 1


def test_product_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_1605_05773_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "d8_oracle" not in text, f
                assert "import cpuref" not in text and "d8_cpuref" not in text, f
