"""CPU-side checks of the C ABI: the library builds, loads, and exports every
symbol include/deoct.h declares (no compute call: no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "deoct.h")).read()
    return sorted(set(re.findall(r"DEOCT_API\s+(?:const\s+char\*|int)\s+(deoct_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_06952_gb300 import build
    return build.build()


def test_header_declares_the_api():
    names = _declared()
    for want in ["deoct_encode", "deoct_eval_population", "deoct_de_step", "deoct_fit_subtree",
                 "deoct_fit_moving_horizon"]:
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2311_06952_gb300 import deoct
    assert sorted(deoct.EXPORTED) == _declared()


def test_version_and_error_string_without_gpu(libpath):
    from paper_2311_06952_gb300 import deoct
    assert "sm_103a" in deoct.version()
    lib = deoct.load()
    # a NULL context is rejected on the host, before any CUDA call
    assert lib.deoct_set_timing(None, 1) == deoct.DEOCT_ERR_INVALID
    assert b"context" in lib.deoct_last_error_string()
    for call in (lambda: lib.deoct_set_scratch_limit(None, 1 << 20), lambda: lib.deoct_release_scratch(None),
                 lambda: lib.deoct_set_eval_config(None, 0, 0, 0, 0),
                 lambda: lib.deoct_set_eval_streaming(None, 1)):
        assert call() == deoct.DEOCT_ERR_INVALID


def test_struct_layouts_match_header():
    from paper_2311_06952_gb300 import deoct
    # deoct_dataset: ptr,int32(+4 pad),int64,ptr,ptr,int64,int32,int32 -> 56 bytes on LP64
    assert ctypes.sizeof(deoct.Dataset) == 56
    # deoct_params: 4 x int32, 2 x float, double, int32, uint32, uint64 -> 48 bytes
    assert ctypes.sizeof(deoct.Params) == 48
    assert ctypes.sizeof(deoct.Stats) == 32


def test_oracle_builds():
    import oracle
    assert os.path.exists(oracle.build())
